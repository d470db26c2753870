"""dri_upload_reference: an uploaded model prediction (world-frame vertex and
normal maps + intensity at a pose) replaces the reference; the systems and the
tracked pose match the oracle's reference_from_upload on the same maps."""
import numpy as np
import pytest

from oracle import maps
from oracle.so3 import State, boxplus, quat_mul
from paper_2207_10940_gb300 import dri, synth
from parity import POSE_M, POSE_RAD, pose_error
from test_gpu_parity import _compare_linearisation, _pair_setup

pytestmark = pytest.mark.gpu


def _prediction(seq, ocfg, frame, x):
    """Frame `frame`'s own level-0 maps moved into W with state x: the maps a
    model rendered at x's pose would give (float32, as uploaded)."""
    lv = maps.frame_levels(seq.depth[frame], seq.intensity[frame], ocfg)[0]
    V_W = (lv.V @ x.R.T + x.r).astype(np.float32)
    N_W = (np.where(lv.N_valid[..., None], lv.N, 0.0) @ x.R.T).astype(np.float32)
    I = np.ascontiguousarray(seq.intensity[frame], dtype=np.float32)
    T = np.concatenate([x.r, x.q])
    return np.ascontiguousarray(V_W), np.ascontiguousarray(N_W), I, T


def _upload(st, tr, ocfg, V_W, N_W, I, T, x, device=False):
    if device:
        import torch
        dev = torch.device("cuda")
        args = [torch.from_numpy(a).to(dev) for a in (V_W, N_W, I)]
        torch.cuda.synchronize()
        dri.dri_upload_reference(st.handle, *args, T)
        torch.cuda.synchronize()
    else:
        dri.dri_upload_reference(st.handle, V_W, N_W, I, T)
    tr.set_reference(maps.reference_from_upload(V_W, N_W, I, x.R, x.r, ocfg), x.R, x.r)


def _compose(a, b):
    """The state whose pose is a's pose followed by b's (b taken relative to W)."""
    x = b.copy()
    x.q = np.asarray(quat_mul(a.q, b.q))
    x.r = a.R @ b.r + a.r
    return x


@pytest.mark.parametrize("device", [False, True])
def test_uploaded_reference_linearisation_matches_oracle(device):
    seq = synth.frame_pair(seed=1)
    st, tr, ocfg, _ = _pair_setup(seq, 2, (10, 5))
    gt0, gt1 = State.from_dict(seq.gt[0]), State.from_dict(seq.gt[1])
    # the prediction: frame 0's view rendered at a pose x_ref away from W's origin,
    # so the transform into the reference camera is not the identity; the live
    # frame 1 then sits at x_ref followed by the true frame 0 -> 1 motion
    xr = boxplus(gt0, np.r_[np.array([0.2, -0.1, 0.15]), np.array([0.1, -0.2, 0.15]), np.zeros(11)])
    V_W, N_W, I, T = _prediction(seq, ocfg, 0, xr)
    _upload(st, tr, ocfg, V_W, N_W, I, T, xr, device)
    x1 = _compose(xr, gt1)
    rng = np.random.default_rng(5)
    for x0, x1 in [(xr, x1), (boxplus(xr, rng.normal(size=17) * 1e-3),
                              boxplus(x1, rng.normal(size=17) * 3e-3))]:
        for level in range(2):
            out, lin = _compare_linearisation(st, tr, seq, ocfg, level, x0, x1)
            assert lin["n_icp"] > 50 and lin["n_rgb"] > 50
    st.close()


def test_tracking_against_an_uploaded_reference_matches_oracle():
    seq = synth.frame_pair(seed=1)
    st, tr, ocfg, _ = _pair_setup(seq, 2, (10, 5))
    gt0 = State.from_dict(seq.gt[0])
    V_W, N_W, I, T = _prediction(seq, ocfg, 0, gt0)       # frame 0 re-rendered at its pose
    _upload(st, tr, ocfg, V_W, N_W, I, T, gt0)
    res = dri.dri_track(st.handle)
    ores = tr.track(seq.depth[1], seq.intensity[1], seq.frame_times[1])
    assert res.status == 0
    da, dr = pose_error(res.x1, ores["x1"])
    assert da < POSE_RAD and dr < POSE_M, (da, dr)
    st.close()


def test_upload_before_the_first_frame_is_not_ready():
    seq = synth.frame_pair(seed=2, cam=synth.scaled_camera(64, 48))
    cfg = dri.dri_config_default(64, 48)
    x = dri.state_from_dict(synth.initial_state(seq))
    h = dri.dri_create_stream(cfg, x)
    V = np.zeros((48, 64, 3), np.float32)
    I = np.zeros((48, 64), np.float32)
    with pytest.raises(dri.DriError) as e:
        dri.dri_upload_reference(h, V, V, I, [0, 0, 0, 1, 0, 0, 0])
    assert e.value.code == dri.DRI_ENOTREADY
    dri.dri_destroy_stream(h)
