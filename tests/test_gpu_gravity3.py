"""The 3-D gravity-with-gauge form of the state on the GPU (gravity_dof =
DRI_GRAVITY_3D; Sec. II and IV-A keep q_IW with three degrees of freedom)
against the oracle's form of it (oracle/gravity3.py): 18 tangent dimensions per
state, the Gauss-Newton step damped on the gravity components of both states,
the undamped system marginalised into an 18 x 18 prior."""
import numpy as np
import pytest

from oracle import gravity3
from oracle.so3 import log_so3
from paper_2207_10940_gb300 import dri, synth
from parity import POSE_M, POSE_RAD, configs, new_stream, pose_error, to_oracle

pytestmark = pytest.mark.gpu
G3 = dri.DRI_GRAVITY_3D


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _gravity_angle(a, b):
    return float(np.linalg.norm(log_so3(a.Rg @ b.Rg.T)))


def _streams(seq, levels, iters, imu_mode=0):
    ocfg, dcfg = configs(seq, levels, iters, imu_mode=imu_mode)
    dcfg.gravity_dof = G3
    x_init = synth.initial_state(seq)
    st = new_stream(dcfg, x_init)
    dri.dri_push_imu(st.handle, seq.imu)
    tr = gravity3.Tracker(ocfg, x_init)
    tr.push_imu(seq.imu)
    return st, tr


@pytest.mark.parametrize("imu_mode", [0, 1])
def test_pair_matches_the_oracle_form(imu_mode):
    _torch()
    seq = synth.frame_pair(seed=1)
    st, tr = _streams(seq, 2, (10, 5), imu_mode)
    for i in range(2):
        dri.dri_upload_frame(st.handle, seq.frame_times[i], seq.depth[i], seq.intensity[i])
        res = dri.dri_track(st.handle)
        ores = tr.track(seq.depth[i], seq.intensity[i], seq.frame_times[i])
        assert res.status == 0
    da, dr = pose_error(res.x1, ores["x1"])
    assert da < POSE_RAD and dr < POSE_M, (da, dr)
    x1 = to_oracle(res.x1)
    np.testing.assert_allclose(x1.v, ores["x1"].v, atol=1e-5)
    np.testing.assert_allclose(x1.bg, ores["x1"].bg, atol=1e-6)
    np.testing.assert_allclose(x1.ba, ores["x1"].ba, atol=1e-5)
    assert _gravity_angle(x1, ores["x1"]) < 1e-6
    # the 18 x 18 prior, on the scale of the system it is the Schur complement of
    _, Hs, bs = dri.dri_get_state(st.handle, with_prior=True)
    assert Hs.shape == (18, 18) and bs.shape == (18,)
    d1 = np.sqrt(np.diag(ores["H"])[18:])
    r = np.max(np.abs(Hs - ores["H_prior"]) / np.outer(d1, d1))
    assert r <= 1e-5, r
    st.close()


def test_sequence_matches_the_oracle_form():
    _torch()
    seq = synth.sinusoid_sequence(seed=4, cam=synth.scaled_camera(160, 120), n_frames=5)
    st, tr = _streams(seq, 3, (6, 4, 3))
    for i in range(5):
        dri.dri_upload_frame(st.handle, seq.frame_times[i], seq.depth[i], seq.intensity[i])
        res = dri.dri_track(st.handle)
        ores = tr.track(seq.depth[i], seq.intensity[i], seq.frame_times[i])
        assert res.status == 0
        if i:
            da, dr = pose_error(res.x1, ores["x1"])
            assert da < 5 * POSE_RAD and dr < 5 * POSE_M, (i, da, dr)
            # The rest of the state along the estimate's own information: over a
            # few frames gravity's tilt and the accelerometer bias trade off (a
            # tilt of 5e-6 rad is 5e-5 m/s^2 of bias) and the turn about gravity
            # is held only by the priors and the damping, so FP32-level
            # differences of the pixel systems move the two solutions apart
            # along those weakly observed directions.  Their difference, in the
            # metric of the oracle's 18 x 18 information H* of x1, stays below
            # 1% of one standard deviation (measured 0.002 at the fourth frame,
            # as much of it from the poses' 5e-6 as from the rest).
            d = gravity3.boxminus(to_oracle(res.x1), ores["x1"])
            m = float(np.sqrt(d @ ores["H_prior"] @ d))
            assert m < 1e-2, (i, m)
    st.close()


def test_batch_mixing_both_forms_equals_each_alone():
    """A 2-DoF and a 3-D stream tracked in one batch give the states each gets
    tracked alone (rows per thread fixed, so the pixel sums are the same)."""
    torch = _torch()
    seq = synth.sinusoid_sequence(seed=8, cam=synth.scaled_camera(160, 120), n_frames=4)
    x_init = synth.initial_state(seq)
    ts = torch.cuda.Stream()

    def make(g):
        _, dcfg = configs(seq, 3, (4, 3, 2))
        dcfg.gravity_dof = g
        st = dri.Stream(dcfg, dri.state_from_dict(x_init), ts)
        dri.dri_push_imu(st.handle, seq.imu)
        return st

    alone = {}
    for g in (dri.DRI_GRAVITY_2DOF, G3):
        st = make(g)
        dri.dri_batch_set_options([st.handle], rows_per_thread=(4, 4, 4))
        for i in range(4):
            dri.dri_upload_frame(st.handle, seq.frame_times[i], seq.depth[i], seq.intensity[i])
            assert dri.dri_track(st.handle).status == 0
        alone[g] = dri.state_to_dict(dri.dri_get_state(st.handle))
        st.close()
    pair = [make(dri.DRI_GRAVITY_2DOF), make(G3)]
    dri.dri_batch_set_options(pair, rows_per_thread=(4, 4, 4), groups=1)
    for i in range(4):
        for st in pair:
            dri.dri_upload_frame(st.handle, seq.frame_times[i], seq.depth[i], seq.intensity[i])
        assert all(r.status == 0 for r in dri.dri_track_batch(pair))
    for st, g in zip(pair, (dri.DRI_GRAVITY_2DOF, G3)):
        got = dri.state_to_dict(dri.dri_get_state(st.handle))
        for k in ("r_WC", "q_WC", "v_I", "q_IW"):
            np.testing.assert_allclose(got[k], alone[g][k], rtol=0, atol=1e-9, err_msg=f"{g} {k}")
        st.close()


def test_linearise_is_not_served_for_the_3d_form():
    _torch()
    seq = synth.frame_pair(seed=2, cam=synth.scaled_camera(64, 48))
    st, _ = _streams(seq, 2, (2, 2))
    for i in range(2):
        dri.dri_upload_frame(st.handle, seq.frame_times[i], seq.depth[i], seq.intensity[i])
        if i == 0:
            dri.dri_track(st.handle)
    x = dri.dri_get_state(st.handle)
    with pytest.raises(dri.DriError) as e:
        dri.dri_linearise(st.handle, 0, x, x)
    assert e.value.code == dri.DRI_EINVAL
    st.close()
