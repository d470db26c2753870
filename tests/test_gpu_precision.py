"""Precision variants of the pixel path against the FP64 oracle.

* DRI_FP32_PARTIALS: per-block partial sums and their fold in FP32 instead of FP64;
* DRI_FP16_MAPS: normals and intensity gradients stored in FP16, gated against an
  oracle that stores its maps in FP16 too (the exact oracle's error is reported
  by bench.py's precision study); the kernel rounds FP32-computed values and the
  oracle FP64-computed ones, which may round to neighbouring half-precision
  values, so this variant's bar is one half-precision unit (2^-11) on the
  normalised systems and 1e-5 rad / 1e-5 m on the pose;
* both.
Every variant keeps FP32 per-pixel arithmetic and the FP64 solve.  The bar is
otherwise the one of the FP32/FP64 path: correspondence validity per pixel
outside the oracle's margins, normalised J^T J / J^T r errors <= 1e-5, final
pose within 1e-6 rad / 1e-6 m.
"""
import numpy as np
import pytest

from oracle.so3 import State, boxplus
from paper_2207_10940_gb300 import dri, synth
from parity import POSE_FP16, POSE_M, POSE_RAD, REL, REL_FP16, pose_error
from test_gpu_parity import _compare_linearisation, _pair_setup

pytestmark = pytest.mark.gpu

VARIANTS = [dri.DRI_FP32_PARTIALS, dri.DRI_FP16_MAPS, dri.DRI_FP16_MAPS | dri.DRI_FP32_PARTIALS]


@pytest.mark.parametrize("flags", VARIANTS)
def test_variant_linearisation_matches_oracle(flags):
    seq = synth.frame_pair(seed=1)
    st, tr, ocfg, dcfg = _pair_setup(seq, 2, (10, 5), precision_flags=flags)
    assert ocfg.fp16_maps == bool(flags & dri.DRI_FP16_MAPS)
    rng = np.random.default_rng(11)
    gt0, gt1 = State.from_dict(seq.gt[0]), State.from_dict(seq.gt[1])
    for x0, x1 in [(gt0, gt1), (boxplus(gt0, rng.normal(size=17) * 1e-3),
                                boxplus(gt1, rng.normal(size=17) * 5e-3))]:
        for level in range(2):
            _compare_linearisation(st, tr, seq, ocfg, level, x0, x1,
                                   rel=REL_FP16 if flags & dri.DRI_FP16_MAPS else REL)
    st.close()


@pytest.mark.parametrize("flags", VARIANTS)
def test_variant_track_pair_matches_oracle(flags):
    seq = synth.frame_pair(seed=1)
    st, tr, ocfg, dcfg = _pair_setup(seq, 2, (10, 5), precision_flags=flags)
    res = dri.dri_track(st.handle)
    ores = tr.track(seq.depth[1], seq.intensity[1], seq.frame_times[1])
    assert res.status == 0
    da, dr = pose_error(res.x1, ores["x1"])
    bar_rad, bar_m = (POSE_FP16, POSE_FP16) if flags & dri.DRI_FP16_MAPS else (POSE_RAD, POSE_M)
    assert da < bar_rad and dr < bar_m, (da, dr)
    st.close()
