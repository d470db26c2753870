"""DRI_IMU_FIRST_ORDER (Forster et al.'s first-order bias update of the
pre-integration instead of re-integrating every iteration) against the oracle's
imu_mode 1, and its reduction to re-integration."""
import numpy as np
import pytest

from oracle import gn
from paper_2207_10940_gb300 import dri, synth
from parity import POSE_M, POSE_RAD, configs, new_stream, pose_error

pytestmark = pytest.mark.gpu


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _track(seq, dcfg, n):
    x_init = synth.initial_state(seq)
    st = new_stream(dcfg, x_init)
    dri.dri_push_imu(st.handle, seq.imu)
    out = []
    for i in range(n):
        dri.dri_upload_frame(st.handle, seq.frame_times[i], seq.depth[i], seq.intensity[i])
        res = dri.dri_track(st.handle)
        assert res.status == 0
        out.append(res)
    x, H, b = dri.dri_get_state(st.handle, with_prior=True)
    st.close()
    return out, x, H, b


def test_first_order_sequence_matches_oracle():
    _torch()
    seq = synth.sinusoid_sequence(seed=4, cam=synth.scaled_camera(160, 120), n_frames=5)
    ocfg, dcfg = configs(seq, 3, (6, 4, 3), imu_mode=dri.DRI_IMU_FIRST_ORDER)
    res, _, _, _ = _track(seq, dcfg, 5)
    tr = gn.Tracker(ocfg, synth.initial_state(seq))
    tr.push_imu(seq.imu)
    for i in range(5):
        ores = tr.track(seq.depth[i], seq.intensity[i], seq.frame_times[i])
        if i:
            da, dr = pose_error(res[i].x1, ores["x1"])
            assert da < 5 * POSE_RAD and dr < 5 * POSE_M, (i, da, dr)


def test_first_order_with_zero_thresholds_is_reintegration_bit_for_bit():
    """Re-integrating whenever the biases move leaves the first iteration of a
    frame (zero bias change, an exact update) as the only first-order one."""
    _torch()
    seq = synth.sinusoid_sequence(seed=5, cam=synth.scaled_camera(96, 72), n_frames=3)
    _, d0 = configs(seq, 2, (4, 3))
    _, d1 = configs(seq, 2, (4, 3), imu_mode=dri.DRI_IMU_FIRST_ORDER, bias_relin_g=0.0,
                    bias_relin_a=0.0)
    _, xa, Ha, ba = _track(seq, d0, 3)
    _, xb, Hb, bb = _track(seq, d1, 3)
    for f in ("r_WC", "q_WC", "v_I", "bg", "ba", "q_IW"):
        assert list(getattr(xa, f)) == list(getattr(xb, f)), f
    assert np.array_equal(Ha, Hb) and np.array_equal(ba, bb)


def test_imu_mode_validation():
    _torch()
    seq = synth.frame_pair(seed=2, cam=synth.scaled_camera(64, 48))
    for kw in (dict(imu_mode=2), dict(imu_mode=1, bias_relin_g=-1.0),
               dict(imu_mode=1, bias_relin_a=float("nan"))):
        _, dcfg = configs(seq, 2, (3, 2), **{k: v for k, v in kw.items()})
        with pytest.raises(dri.DriError) as e:
            new_stream(dcfg, synth.initial_state(seq))
        assert e.value.code == dri.DRI_EINVAL
