"""DRI_TRACK_RGBD_ONLY (the vision-only, pose-only baseline the paper compares
with) against the oracle's track_mode 1, alone and in a batch beside an
RGB-D-inertial stream."""
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


def test_pose_only_sequence_matches_oracle_without_imu():
    _torch()
    seq = synth.sinusoid_sequence(seed=4, cam=synth.scaled_camera(160, 120), n_frames=5)
    ocfg, dcfg = configs(seq, 3, (6, 4, 3), track_mode=dri.DRI_TRACK_RGBD_ONLY, rgbd_lambda=0.5)
    x_init = synth.initial_state(seq)
    st = new_stream(dcfg, x_init)                      # no IMU samples pushed
    tr = gn.Tracker(ocfg, x_init)
    for i in range(5):
        dri.dri_upload_frame(st.handle, seq.frame_times[i], seq.depth[i], seq.intensity[i])
        res = dri.dri_track(st.handle)
        ores = tr.track(seq.depth[i], seq.intensity[i], seq.frame_times[i])
        assert res.status == 0
        if i:
            da, dr = pose_error(res.x1, ores["x1"])
            assert da < (i + 1) * POSE_RAD and dr < (i + 1) * POSE_M, (i, da, dr)
            for f in ("v_I", "bg", "ba"):               # carried over unchanged
                assert list(getattr(res.x1, f)) == list(getattr(res.x0, f)), f
            # the gravity quaternion is renormalised by every state update
            assert np.allclose(list(res.x1.q_IW), list(res.x0.q_IW), rtol=0, atol=1e-15)
    st.close()


def test_mixed_batch_equals_each_stream_alone():
    torch = _torch()
    seq = synth.sinusoid_sequence(seed=7, cam=synth.scaled_camera(96, 72), n_frames=3)
    _, d_in = configs(seq, 2, (4, 3))
    _, d_rg = configs(seq, 2, (4, 3), track_mode=dri.DRI_TRACK_RGBD_ONLY)
    x_init = synth.initial_state(seq)

    def run(cfgs, batched):
        ts = torch.cuda.Stream()
        sts = [dri.Stream(c, dri.state_from_dict(x_init, 0.0), ts) for c in cfgs]
        for st in sts:
            dri.dri_push_imu(st.handle, seq.imu)
        for i in range(3):
            for st in sts:
                dri.dri_upload_frame(st.handle, seq.frame_times[i], seq.depth[i], seq.intensity[i])
            if batched:
                dri.dri_track_batch(sts, wait=True)
            else:
                for st in sts:
                    dri.dri_track(st.handle)
        out = [dri.dri_get_state(st.handle) for st in sts]
        for st in sts:
            st.close()
        return out

    alone = run([d_in], False) + run([d_rg], False)
    mixed = run([d_in, d_rg], True)
    for a, b in zip(alone, mixed):
        da, dr = pose_error(a, b)
        assert da < POSE_RAD and dr < POSE_M, (da, dr)
    # the two modes really differ
    da, dr = pose_error(mixed[0], mixed[1])
    assert da + dr > 1e-5


def test_track_mode_validation():
    _torch()
    seq = synth.frame_pair(seed=2, cam=synth.scaled_camera(64, 48))
    for kw in (dict(track_mode=3), dict(track_mode=-1), dict(track_mode=1, rgbd_lambda=-1.0)):
        _, dcfg = configs(seq, 2, (3, 2), **kw)
        with pytest.raises(dri.DriError) as e:
            new_stream(dcfg, synth.initial_state(seq))
        assert e.value.code == dri.DRI_EINVAL
