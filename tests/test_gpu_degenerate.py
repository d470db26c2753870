"""Degenerate inputs of the method against the oracle.

* Textureless frames (the paper's counter-example of a camera facing a white
  wall, Sec. V): constant intensity makes every photometric Jacobian exactly
  zero (zero image gradient, Eq. 3), so the photometric system is exactly zero
  on both sides and only the ICP and IMU terms constrain the step.
* A static camera: zero rotation and translation over the frame interval (the
  IMU measures gravity and the biases only); the tracker must stay put as the
  oracle does."""
import copy

import numpy as np
import pytest

from paper_2207_10940_gb300 import dri, synth
from parity import POSE_M, POSE_RAD, pose_error, to_oracle
from test_gpu_parity import _compare_linearisation, _pair_setup

pytestmark = pytest.mark.gpu


def _textureless(seq, value=0.5):
    seq.intensity = [np.full_like(i, value) for i in seq.intensity]
    return seq


def test_textureless_frames_match_oracle():
    seq = _textureless(synth.frame_pair(seed=2))
    st, tr, ocfg, _ = _pair_setup(seq, 2, (10, 5))
    before = copy.deepcopy(tr)
    ores = tr.track(seq.depth[1], seq.intensity[1], seq.frame_times[1])
    for level in (1, 0):
        x0, x1 = ores["points"][level]
        out, lin = _compare_linearisation(st, before, seq, ocfg, level, x0, x1)
        # valid photometric correspondences with an exactly zero system
        assert lin["n_rgb"] > 0 and not np.any(lin["H_rgb"])
        assert not np.any(np.array(out.H_rgb)) and not np.any(np.array(out.b_rgb))
    res = dri.dri_track(st.handle)
    assert res.status == 0
    da, dr = pose_error(res.x1, ores["x1"])
    assert da < POSE_RAD and dr < POSE_M, (da, dr)
    st.close()


def test_static_camera_matches_oracle():
    seq = synth.frame_pair(seed=5, rot_deg=0.0, trans_m=0.0)
    st, tr, ocfg, _ = _pair_setup(seq, 2, (10, 5))
    res = dri.dri_track(st.handle)
    ores = tr.track(seq.depth[1], seq.intensity[1], seq.frame_times[1])
    assert res.status == 0
    da, dr = pose_error(res.x1, ores["x1"])
    assert da < POSE_RAD and dr < POSE_M, (da, dr)
    x1 = to_oracle(res.x1)
    np.testing.assert_allclose(x1.v, ores["x1"].v, atol=1e-5)
    # the estimate stays close to the (static) ground truth
    gt1 = seq.gt[1]
    assert np.linalg.norm(x1.r - np.asarray(gt1["r_WC"])) < 5e-3
    st.close()
