"""The depth-dependent ICP weight (icp_depth_weight = 1: W_ICP / z^4), alone and
with the occlusion test, against the oracle: per-pixel validity outside the
margins, the systems, a tracked sequence; batches must agree on it."""
import numpy as np
import pytest

from oracle import gn
from oracle.so3 import State, boxplus
from paper_2207_10940_gb300 import dri, synth
from parity import POSE_M, POSE_RAD, configs, new_stream, pose_error
from test_gpu_parity import _compare_linearisation, _pair_setup

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("occ", [0.0, 0.03])
def test_linearisation_with_depth_weight_matches_oracle(occ):
    seq = synth.frame_pair(seed=1, cam=synth.CAM_320, trans_m=0.08)
    st, tr, ocfg, _ = _pair_setup(seq, 2, (10, 5), icp_depth_weight=1, occlusion_thr=occ)
    rng = np.random.default_rng(2)
    gt0, gt1 = State.from_dict(seq.gt[0]), State.from_dict(seq.gt[1])
    for x0, x1 in [(gt0, gt1),
                   (boxplus(gt0, rng.normal(size=17) * 1e-3), boxplus(gt1, rng.normal(size=17) * 5e-3))]:
        for level in range(2):
            _, lin = _compare_linearisation(st, tr, seq, ocfg, level, x0, x1)
            assert lin["n_icp"] > 50
    st.close()


def test_tracking_with_depth_weight_matches_oracle():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    seq = synth.sinusoid_sequence(seed=4, cam=synth.scaled_camera(160, 120), n_frames=4)
    ocfg, dcfg = configs(seq, 3, (6, 4, 3), icp_depth_weight=1)
    x_init = synth.initial_state(seq)
    st = new_stream(dcfg, x_init)
    dri.dri_push_imu(st.handle, seq.imu)
    tr = gn.Tracker(ocfg, x_init)
    tr.push_imu(seq.imu)
    for i in range(4):
        dri.dri_upload_frame(st.handle, seq.frame_times[i], seq.depth[i], seq.intensity[i])
        res = dri.dri_track(st.handle)
        ores = tr.track(seq.depth[i], seq.intensity[i], seq.frame_times[i])
        assert res.status == 0
        if i:
            da, dr = pose_error(res.x1, ores["x1"])
            assert da < (i + 1) * POSE_RAD and dr < (i + 1) * POSE_M, (i, da, dr)
    st.close()


def test_batch_must_agree_on_the_depth_weight_and_its_validation():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    seq = synth.frame_pair(seed=2, cam=synth.scaled_camera(64, 48))
    _, a = configs(seq, 2, (3, 2))
    _, b = configs(seq, 2, (3, 2), icp_depth_weight=1)
    ts = torch.cuda.Stream()
    sa = dri.Stream(a, dri.state_from_dict(synth.initial_state(seq), 0.0), ts)
    sb = dri.Stream(b, dri.state_from_dict(synth.initial_state(seq), 0.0), ts)
    for s in (sa, sb):
        dri.dri_upload_frame(s.handle, seq.frame_times[0], seq.depth[0], seq.intensity[0])
    with pytest.raises(dri.DriError) as e:
        dri.dri_track_batch([sa, sb], wait=True)
    assert e.value.code == dri.DRI_EINVAL
    sa.close()
    sb.close()
    _, c = configs(seq, 2, (3, 2), icp_depth_weight=2)
    with pytest.raises(dri.DriError) as e:
        new_stream(c, synth.initial_state(seq))
    assert e.value.code == dri.DRI_EINVAL
