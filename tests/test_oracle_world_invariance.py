"""Invariance of the pixel terms (Eq. 3-4) to the choice of world frame: moving
the whole scene description rigidly -- the reference pose, its world-frame maps
and both states by the same rotation R_G and translation t_G -- changes no
residual, cost or correspondence, and turns the world-frame systems by
Q = diag(R_G, R_G) with no translation coupling (the rotation Jacobians use
camera-centred points s = R p, Sec. IV-B).  A Jacobian taken about the world
origin, or a rotation applied on the wrong side, fails this."""
import numpy as np
import pytest

from conftest import oracle_config
from oracle.maps import frame_levels, reference_from_frame
from oracle.photogeo import linearise
from oracle.so3 import State, boxplus, exp_so3, rot_to_quat
from paper_2207_10940_gb300 import synth


def _move(x, RG, tG):
    y = x.copy()
    y.q = rot_to_quat(RG @ x.R)
    y.r = RG @ x.r + tG
    return y


@pytest.mark.parametrize("seed", [1, 2])
def test_pixel_terms_do_not_depend_on_the_world_frame(seed):
    seq = synth.frame_pair(seed=seed, cam=synth.scaled_camera(64, 48))
    cfg = oracle_config(seq, levels=2)
    rng = np.random.default_rng(40 + seed)
    g0, g1 = State.from_dict(seq.gt[0]), State.from_dict(seq.gt[1])
    x0 = boxplus(g0, rng.normal(size=17) * 2e-3)
    x1 = boxplus(g1, rng.normal(size=17) * 4e-3)
    RG = exp_so3(rng.normal(size=3))
    tG = rng.normal(size=3)
    lv0 = frame_levels(seq.depth[0], seq.intensity[0], cfg)
    lv1 = frame_levels(seq.depth[1], seq.intensity[1], cfg)
    R_ref, r_ref = g0.R, g0.r
    ref = reference_from_frame(lv0, R_ref, r_ref)
    ref_g = reference_from_frame(lv0, RG @ R_ref, RG @ r_ref + tG)
    Q = np.zeros((6, 6))
    Q[:3, :3] = Q[3:, 3:] = RG
    Q2 = np.zeros((12, 12))
    Q2[:6, :6] = Q2[6:, 6:] = Q
    for level in range(2):
        a = linearise(lv1[level], ref[level], R_ref, r_ref, x0, x1, cfg)
        b = linearise(lv1[level], ref_g[level], RG @ R_ref, RG @ r_ref + tG, _move(x0, RG, tG),
                      _move(x1, RG, tG), cfg)
        assert np.array_equal(a["icp_valid"], b["icp_valid"])
        assert np.array_equal(a["rgb_valid"], b["rgb_valid"])
        assert a["n_icp"] > 50 and a["n_rgb"] > 50
        for k in ("cost_icp", "cost_rgb"):
            assert abs(a[k] - b[k]) <= 1e-9 * a[k], k
        for H, g, QQ in (("H_icp", "b_icp", Q), ("H_rgb", "b_rgb", Q2)):
            s = np.abs(a[H]).max()
            np.testing.assert_allclose(b[H], QQ @ a[H] @ QQ.T, rtol=0, atol=1e-9 * s, err_msg=H)
            sb = np.sqrt(s * (a["cost_icp"] + a["cost_rgb"]))
            np.testing.assert_allclose(b[g], QQ @ a[g], rtol=0, atol=1e-9 * sb, err_msg=g)
