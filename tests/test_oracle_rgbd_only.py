"""Pins of the oracle's RGB-D-only baseline (track_mode 1: the vision-only,
pose-only tracker the paper compares with, Sec. III)."""
import numpy as np

from conftest import oracle_config
from oracle import gn
from oracle.maps import frame_levels
from oracle.photogeo import linearise
from oracle.so3 import State, log_so3
from paper_2207_10940_gb300 import synth


def _tracker(seq, **kw):
    cfg = oracle_config(seq, levels=2, iters=(8, 5), track_mode=1, **kw)
    tr = gn.Tracker(cfg, synth.initial_state(seq))
    tr.track(seq.depth[0], seq.intensity[0], seq.frame_times[0])
    return tr, cfg


def test_no_motion_noise_free_keeps_the_pose():
    """Identical frames: the residuals vanish up to the rounding of rebuilding
    the reference vertex from its depth (~1e-17 m), so the pose stays put."""
    seq = synth.frame_pair(seed=6, cam=synth.scaled_camera(48, 36), rot_deg=0.0, trans_m=0.0,
                           sigma_d=0.0, sigma_I=0.0, imu_noise=False)
    tr, _ = _tracker(seq)
    x0 = tr.x.copy()
    r = tr.track(seq.depth[1], seq.intensity[1], seq.frame_times[1])
    assert np.linalg.norm(r["x1"].r - x0.r) < 1e-12
    assert np.linalg.norm(log_so3(r["x1"].R @ x0.R.T)) < 1e-12


def test_converges_to_the_true_motion_noise_free():
    seq = synth.frame_pair(seed=3, cam=synth.scaled_camera(96, 72), sigma_d=0.0, sigma_I=0.0,
                           imu_noise=False)
    tr, _ = _tracker(seq)
    r = tr.track(seq.depth[1], seq.intensity[1], seq.frame_times[1])
    g = State.from_dict(seq.gt[1])
    # 2 deg / 3 cm of motion recovered to well under a pixel's worth
    assert np.linalg.norm(log_so3(r["x1"].R @ g.R.T)) < 2e-3
    assert np.linalg.norm(r["x1"].r - g.r) < 5e-3


def test_cost_decreases_and_only_the_pose_moves():
    seq = synth.frame_pair(seed=3, cam=synth.scaled_camera(64, 48))
    tr, cfg = _tracker(seq, rgbd_lambda=0.5)
    x0 = tr.x.copy()
    ref, T_ref = tr.ref, tr.T_ref
    lv = frame_levels(seq.depth[1], seq.intensity[1], cfg)

    def cost(x1):
        lin = linearise(lv[0], ref[0], T_ref[0], T_ref[1], x0, x1, cfg)
        return lin["cost_icp"] + cfg.rgbd_lambda * lin["cost_rgb"]

    r = tr.track(seq.depth[1], seq.intensity[1], seq.frame_times[1])
    assert cost(r["x1"]) < 0.5 * cost(x0)
    for f in ("v", "bg", "ba", "qg"):
        assert np.array_equal(getattr(r["x1"], f), getattr(x0, f)), f
