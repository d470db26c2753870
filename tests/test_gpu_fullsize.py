"""The pixel kernel that tracking runs (the batched kernel, through the stream's
own one-slot plan) against the FP64 oracle at the benchmark's image sizes.

dri_linearise evaluates the pixel terms with the same batched kernel and rows
per thread that dri_track / dri_track_batch launch, so these tests compare the
production kernel with the oracle per pixel and per system entry:

* 640x480 with 32 / 32 / 8 rows per thread (the benchmark's tiles: 8,192
  pixels summed in FP32 per thread group before the FP64 partial) and
  1280x720 with 32 / 16 / 8, both with 1% of the depth pixels dropped (holes
  that exercise depth validity in the pyramid, the normals and association);
* at the oracle's last linearisation point of every pyramid level of a tracked
  frame (Sec. IV-D), so the per-pixel validity that the oracle's per-level
  counts come from is checked bit-exactly outside the margin pixels (so is the
  ICP association), and the systems within the 1e-5 normalised bar (Eq. 7)
  plus the bounded contribution of any margin pixel the two decided
  differently (parity.margin_allowance);
* then the frame is tracked and its pose compared within 1e-6 rad / 1e-6 m
  (1e-5 with FP16 maps), the whole state within 10% of one standard deviation
  of the oracle's posterior information.
"""
import copy

import numpy as np
import pytest

from oracle import gn, imu, maps
from oracle.so3 import State, boxminus, boxplus
from paper_2207_10940_gb300 import dri, synth
from parity import (POSE_FP16, POSE_M, POSE_RAD, REL, REL_FP16, compare_linearisation, configs, new_stream,
                    pose_error, to_dri, to_oracle)

pytestmark = pytest.mark.gpu


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _check_level(st, tr, seq, ocfg, level, x0, x1, rel=REL):
    """dri_linearise at (x0, x1) against the oracle tracker `tr` (state before the
    frame): validity and association per pixel outside margins, counts, systems."""
    shape = (ocfg.height >> level, ocfg.width >> level)
    out, flags = dri.dri_linearise(st.handle, level, to_dri(x0), to_dri(x1), want_flags=True, shape=shape)
    lv = maps.frame_levels(seq.depth[1], seq.intensity[1], ocfg)
    t0, t1 = seq.frame_times[0], seq.frame_times[1]
    W, _ = imu.weight(x0, tr.imu, t0, t1, ocfg)
    H, b, parts = tr.linearise_all(lv, level, x0, x1, t0, t1, W)
    lin = parts["lin"]
    d = boxminus(x0, tr.xbar)
    cost = lin["cost_icp"] + lin["cost_rgb"] + parts["cost_imu"] + float(d @ tr.Hs @ d)
    compare_linearisation(out, flags, lin, H, b, cost, lv[level], tr.ref[level], x0, x1, ocfg, rel=rel,
                          what=f"level {level}")
    return lin


def _full_size_case(cam, seed, rows, trans_m=0.03, **options):
    _torch()
    seq = synth.frame_pair(seed=seed, cam=cam, dropout=0.01, trans_m=trans_m)
    assert (seq.depth[1] == 0).mean() > 0.005                 # the holes are there
    ocfg, dcfg = configs(seq, 3, (10, 5, 4), **options)
    fp16 = bool(options.get("precision_flags", 0) & dri.DRI_FP16_MAPS)
    rel, bar = (REL_FP16, POSE_FP16) if fp16 else (REL, None)
    x_init = synth.initial_state(seq)
    st = new_stream(dcfg, x_init)
    dri.dri_batch_set_options([st.handle], rows_per_thread=rows)
    assert list(dri.dri_batch_get_options([st.handle]).rows_per_thread)[:3] == list(rows)
    dri.dri_push_imu(st.handle, seq.imu)
    dri.dri_upload_frame(st.handle, seq.frame_times[0], seq.depth[0], seq.intensity[0])
    assert dri.dri_track(st.handle).initialised == 1
    dri.dri_upload_frame(st.handle, seq.frame_times[1], seq.depth[1], seq.intensity[1])
    tr = gn.Tracker(ocfg, x_init)
    tr.push_imu(seq.imu)
    tr.track(seq.depth[0], seq.intensity[0], seq.frame_times[0])
    before = copy.deepcopy(tr)
    ores = tr.track(seq.depth[1], seq.intensity[1], seq.frame_times[1])
    for level in (2, 1, 0):
        x0, x1 = ores["points"][level]
        lin = _check_level(st, before, seq, ocfg, level, x0, x1, rel)
        assert (lin["n_icp"], lin["n_rgb"]) == ores["counts"][level]
    # a perturbed state at level 0 as well (projections away from the optimum)
    rng = np.random.default_rng(seed)
    gt0, gt1 = State.from_dict(seq.gt[0]), State.from_dict(seq.gt[1])
    _check_level(st, before, seq, ocfg, 0, boxplus(gt0, rng.normal(size=17) * 1e-3),
                 boxplus(gt1, rng.normal(size=17) * 5e-3), rel)
    res = dri.dri_track(st.handle)
    assert res.status == 0
    da, dr = pose_error(res.x1, ores["x1"])
    assert da < (bar or POSE_RAD) and dr < (bar or POSE_M), (da, dr)
    x1 = to_oracle(res.x1)
    # the rest of the state (velocity, biases, gravity) in the metric of the
    # information the frame gives it, the oracle's posterior H* of x1: one frame
    # pair observes the biases weakly, so FP32-level differences of the pixel
    # systems move them along weakly informed directions.  The systems' bar
    # (1e-5 sqrt(H_ii C) per entry of b, C ~ the residual count) alone allows
    # ~1e-5 sqrt(34 C) = 0.03 at 640x480, the margin pixels decided differently
    # more; the whole difference stays below 10% of one standard deviation
    d = boxminus(x1, ores["x1"])
    m = float(np.sqrt(d @ ores["H_prior"] @ d))
    assert m < 0.1, m
    st.close()


def test_production_kernel_matches_oracle_640x480_with_holes():
    _full_size_case(synth.CAM_640, 11, (32, 32, 8))


def test_production_kernel_matches_oracle_1280x720_with_holes():
    _full_size_case(synth.CAM_1280, 12, (32, 16, 8))


# The options at the benchmark's size and tiling: each is a compile-time variant
# of the production pixel kernel (or of its storage and reduction), compared
# with the oracle's matching mode (readings 17, 21, 22 and the FP32-partials
# variant of the precision study) per pixel, per system entry and in tracking.
@pytest.mark.parametrize("name,options", [
    ("fp16_maps", dict(precision_flags=1)),
    ("fp32_partials", dict(precision_flags=2)),
    ("occlusion", dict(occlusion_thr=0.03, trans_m=0.08)),
    ("depth_weight", dict(icp_depth_weight=1)),
])
def test_options_match_oracle_640x480(name, options):
    _full_size_case(synth.CAM_640, 13, (32, 32, 8), **options)
