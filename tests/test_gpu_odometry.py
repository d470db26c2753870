"""Odometry on a synthetic sequence (the paper's Sec. V evaluation, Fig. 3
convergence): the library's trajectory follows the oracle's frame by frame, so
the trajectory errors against ground truth agree too."""
import numpy as np
import pytest

from oracle import gn
from paper_2207_10940_gb300 import dri, odometry, synth
from parity import POSE_M, POSE_RAD, configs, new_stream, pose_error

pytestmark = pytest.mark.gpu

N_FRAMES = 24


def test_trajectory_and_its_errors_match_the_oracle():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    seq = synth.sinusoid_sequence(seed=4, cam=synth.scaled_camera(160, 120), n_frames=N_FRAMES)
    ocfg, dcfg = configs(seq, 3, (6, 4, 3))
    x_init = synth.initial_state(seq)
    st = new_stream(dcfg, x_init)
    dri.dri_push_imu(st.handle, seq.imu)
    tr = gn.Tracker(ocfg, x_init)
    tr.push_imu(seq.imu)
    ours, theirs = [], []
    for i in range(N_FRAMES):
        dri.dri_upload_frame(st.handle, seq.frame_times[i], seq.depth[i], seq.intensity[i])
        res = dri.dri_track(st.handle)
        ores = tr.track(seq.depth[i], seq.intensity[i], seq.frame_times[i])
        assert res.status == 0
        # each frame starts from the previous one's result, so the per-frame
        # bound of the single-frame tests adds up along the chain
        da, dr = pose_error(res.x1, ores["x1"])
        assert da < (i + 1) * POSE_RAD and dr < (i + 1) * POSE_M, (i, da, dr)
        ours.append(dri.state_to_dict(res.x1))
        theirs.append(ores["x1"].to_dict())
    st.close()
    eo, et = odometry.evaluate(ours, seq.gt), odometry.evaluate(theirs, seq.gt)
    for k in ("ate_rmse_m", "ate_rmse_unaligned_m", "final_position_error_m"):
        assert abs(eo[k] - et[k]) <= N_FRAMES * POSE_M, (k, eo[k], et[k])
    assert abs(eo["rotation_rmse_rad"] - et["rotation_rmse_rad"]) <= N_FRAMES * POSE_RAD
    # sanity of the tracker itself (no robust kernel, no occlusion test): it
    # stays within centimetres and a few degrees over the 0.8 s
    assert eo["ate_rmse_m"] < 0.02 and eo["rotation_rmse_rad"] < 0.05
    assert np.isfinite(eo["velocity_rmse_mps"]) and eo["velocity_rmse_mps"] < 0.2
