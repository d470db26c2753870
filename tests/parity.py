"""Shared helpers of the GPU parity tests: matching oracle / library configurations,
state conversions and the tolerance checks of the parity bar.

Tolerances (stated once here, used by every parity test):
* valid-correspondence counts: bit-exact per pixel outside the oracle's margin
  pixels (1e-4 px of a bound or rounding boundary, relative 1e-5 of a threshold);
  the ICP association (the reference pixel) likewise;
* J^T J and J^T r entries: |dH_ij| <= 1e-5 sqrt(H_ii H_jj) and
  |db_i| <= 1e-5 sqrt(H_ii C) with C the cost of the terms in the system, plus,
  for the margin pixels that the kernel decided differently from the oracle
  (validity or association, read from its per-pixel flags), the largest
  contribution such a pixel can make on either side (`margin_allowance`): one
  ICP pixel carries ~1/n of the system, more than 1e-5 of it at these sizes;
* final pose: 1e-6 rad and 1e-6 m.
"""
import numpy as np

from conftest import oracle_config
from oracle.so3 import State, log_so3
from paper_2207_10940_gb300 import dri, synth

REL = 1e-5
POSE_RAD = 1e-6
POSE_M = 1e-6
# FP16-stored normals / gradients: each stored value is exact only to one
# half-precision unit, and an FP32 kernel and the FP64 oracle may round values
# that straddle a rounding boundary to neighbouring units, so the systems agree
# to that unit (2^-11, normalised as above) and the pose to ten times the FP32 bar.
REL_FP16 = 2.0 ** -11
POSE_FP16 = 1e-5


def configs(seq, levels, iters, precision_flags=0, **kw):
    """Matching oracle and library configurations; the oracle stores its maps in
    FP16 exactly when the library does (DRI_FP16_MAPS)."""
    ocfg = oracle_config(seq, levels=levels, iters=iters,
                         fp16_maps=bool(precision_flags & dri.DRI_FP16_MAPS), **kw)
    cam = seq.cam
    dcfg = dri.config_for(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, levels, iters,
                          q_CS=synth.matrix_to_quat(seq.R_CS), r_CS=seq.r_CS,
                          precision_flags=precision_flags, **kw)
    return ocfg, dcfg


def to_dri(x, t=0.0):
    return dri.state_from_dict(x.to_dict() if isinstance(x, State) else x, t)


def to_oracle(x):
    return State.from_dict(dri.state_to_dict(x))


def check_system(H_g, b_g, H_o, b_o, cost, rel=REL, what="", allow=None):
    """allow: optional (A_H, A_b, A_cost) added to the tolerances (margin pixels
    decided differently, `margin_allowance`)."""
    H_g, b_g, H_o, b_o = map(np.asarray, (H_g, b_g, H_o, b_o))
    A_H, A_b, A_c = (0.0, 0.0, 0.0) if allow is None else allow
    d = np.sqrt(np.maximum(np.diag(H_o), 0.0))
    tolH = rel * np.outer(d, d) + A_H
    errH = np.abs(H_g - H_o)
    worst = np.max(errH / np.maximum(tolH, 1e-300))
    assert np.all(errH <= tolH), f"{what} H: worst err/tol {worst:.3g}"
    tolb = rel * np.sqrt(np.maximum(np.diag(H_o), 0.0) * max(cost + A_c, 0.0)) + A_b
    errb = np.abs(b_g - b_o)
    worstb = np.max(errb / np.maximum(tolb, 1e-300))
    assert np.all(errb <= tolb), f"{what} b: worst err/tol {worstb:.3g}"
    return worst, worstb


def decided_differently(lin, flags):
    """Pixels the kernel decided differently from the oracle, from its flag
    bytes (bit 0 ICP valid, bit 1 photometric valid, bits 2-5 the ICP reference
    pixel as x mod 4 | (y mod 4) << 2): (gpu ICP valid, gpu photometric valid,
    ICP differs, photometric differs).  ICP differs where the validity differs
    or both accept with different reference pixels (the two differ by at most
    one pixel, which the residues mod 4 tell apart)."""
    gi, gr = (flags & 1) != 0, (flags & 2) != 0
    oi, orr = lin["icp_valid"], lin["rgb_valid"]
    px = lin["px"]
    both = gi & oi
    o_assoc = np.zeros(flags.shape, dtype=np.int64)
    o_assoc[both] = ((px["xi"][both].astype(np.int64) & 3) |
                     ((px["yi"][both].astype(np.int64) & 3) << 2))
    g_assoc = (flags.astype(np.int64) >> 2) & 15
    d_icp = (gi != oi) | (both & (g_assoc != o_assoc))
    return gi, gr, d_icp, gr != orr


def margin_allowance(lin, flags, cur, ref, x0, x1, cfg):
    """Bounds on what the pixels decided differently can change in the ICP,
    photometric and joint systems, from the oracle's values at those pixels
    and bounds of the kernel's: per pixel, the oracle's own contribution (where
    it accepts) plus the largest a kernel contribution can be (where the
    kernel accepts).  ICP: |J_i| <= |N| (translation rows) and <= |s| |N|
    (rotation rows) with |N| <= 1.001 (FP16 normals), |e| < d_thr; photometric:
    |J_i| <= |a| and <= |s| |a| with |a| <= G (f_x + f_y + |x - c_x| + |y - c_y| + 2) / z_0,
    G the largest stored gradient component, |e| <= max I_0 + max I_1.  Also
    asserts that every such pixel is a margin pixel (per-pixel bar).
    Returns dict(icp=(A_H 6x6, A_b 6, A_cost), rgb=(x1 block), joint=(34x34, 34, cost))."""
    gi, gr, d_icp, d_rgb = decided_differently(lin, flags)
    assert not np.any(d_icp & ~lin["icp_margin"]), \
        f"ICP decided differently at {int((d_icp & ~lin['icp_margin']).sum())} non-margin pixels"
    assert not np.any(d_rgb & ~lin["rgb_margin"]), \
        f"photometric decided differently at {int((d_rgb & ~lin['rgb_margin']).sum())} non-margin pixels"
    W_icp, W_rgb = 1.0 / cfg.sigma_d ** 2, 1.0 / cfg.sigma_I ** 2
    px = lin["px"]
    s_norm = np.linalg.norm(cur.V, axis=-1)        # |s_1| = |R_1 p| = |p|
    dw = bool(getattr(cfg, "icp_depth_weight", 0))
    A_icp, a_icp, c_icp = np.zeros((6, 6)), np.zeros(6), 0.0
    for m in zip(*np.nonzero(d_icp)):
        sc = 1.0 / float(cur.depth[m]) ** 2 if dw else 1.0
        if lin["icp_valid"][m]:
            J, e = px["J_icp"][m] * sc, float(px["e_icp"][m]) * sc
            A_icp += W_icp * np.abs(np.outer(J, J))
            a_icp += W_icp * np.abs(J * e)
            c_icp += W_icp * e * e
        if gi[m]:
            c = 1.001 * np.array([1.0, 1.0, 1.0] + [s_norm[m]] * 3) * sc
            e = cfg.icp_dist_thr * sc
            A_icp += W_icp * np.outer(c, c)
            a_icp += W_icp * c * e
            c_icp += W_icp * e * e
    R0, r0, R1, r1 = x0.R, x0.r, x1.R, x1.r
    M = np.eye(6)
    M[3:, :3] = np.array([[0, -(r1 - r0)[2], (r1 - r0)[1]], [(r1 - r0)[2], 0, -(r1 - r0)[0]],
                          [-(r1 - r0)[1], (r1 - r0)[0], 0]])
    A12, a12, c_rgb = np.zeros((12, 12)), np.zeros(12), 0.0
    if d_rgb.any():
        cam = cur.cam
        G = float(np.max(np.abs(ref.G)))
        e_max = float(np.max(ref.I)) + float(np.max(cur.I))
        p0 = ((cur.V @ R1.T + r1) - r0) @ R0
        for m in zip(*np.nonzero(d_rgb)):
            if lin["rgb_valid"][m]:
                J, e = px["J_rgb"][m], float(px["e_rgb"][m])
                A12 += W_rgb * np.abs(np.outer(J, J))
                a12 += W_rgb * np.abs(J * e)
                c_rgb += W_rgb * e * e
            if gr[m]:
                z0 = max(abs(float(p0[m][2])), 1e-9)
                a = G * (cam["fx"] + cam["fy"] + abs(px["xp"][m] - cam["cx"]) + abs(px["yp"][m] - cam["cy"])
                         + 2.0) / z0
                c1 = np.array([a, a, a] + [s_norm[m] * a] * 3)
                c = np.concatenate([np.abs(M) @ c1, c1])      # J_0 = -M J_1
                A12 += W_rgb * np.outer(c, c)
                a12 += W_rgb * c * e_max
                c_rgb += W_rgb * e_max * e_max
    AJ, aJ = np.zeros((34, 34)), np.zeros(34)
    idx = np.r_[0:6, 17:23]
    AJ[np.ix_(idx, idx)] += A12
    aJ[idx] += a12
    AJ[17:23, 17:23] += A_icp
    aJ[17:23] += a_icp
    return dict(icp=(A_icp, a_icp, c_icp), rgb=(A12[6:, 6:], a12[6:], c_rgb),
                joint=(AJ, aJ, c_icp + c_rgb))


def pose_error(xa, xb):
    """(rotation angle between the two camera orientations, position distance)."""
    a = xa if isinstance(xa, State) else to_oracle(xa)
    b = xb if isinstance(xb, State) else to_oracle(xb)
    return float(np.linalg.norm(log_so3(a.R @ b.R.T))), float(np.linalg.norm(a.r - b.r))


def new_stream(dcfg, x_init):
    import torch
    return dri.Stream(dcfg, to_dri(x_init, x_init.get("t", 0.0) if isinstance(x_init, dict) else 0.0),
                      torch.cuda.Stream())


def check_margins(out, flags, lin, what=""):
    """The kernel's margin decisions (flag bits 6 ICP, 7 photometric): their
    counts equal the bits (the counting and the flag-writing launches are one
    kernel), and per pixel they are the oracle's margins of the decisions the
    linearisation makes (icp_margin_px, rgb_margin_px) except where a pixel's
    margin quantity lies within FP32 rounding of the margin's own edge: a
    pixel's distance to a rounding boundary carries ~1e-6 px of FP32 error, so
    with two edges per axis and two axes about 8e-6 of the pixels sit that
    close to an edge (a Poisson count), and the distance, angle and occlusion
    tests add theirs; bounded here by twice that, max(8, 2e-5 x pixels) per
    term."""
    gm_i, gm_r = (flags & 64) != 0, (flags & 128) != 0
    assert out.n_margin_icp == gm_i.sum() and out.n_margin_rgb == gm_r.sum(), \
        (what, out.n_margin_icp, gm_i.sum(), out.n_margin_rgb, gm_r.sum())
    bar = max(8, 2e-5 * flags.size)
    for name, g, o in (("ICP", gm_i, lin["icp_margin_px"]), ("photometric", gm_r, lin["rgb_margin_px"])):
        diff = int((g != o).sum())
        assert diff <= bar, \
            f"{what} {name} margins: {diff} pixels differ (kernel {g.sum()}, oracle {o.sum()})"


def compare_linearisation(out, flags, lin, H, b, cost, cur, ref, x0, x1, cfg, rel=REL, what=""):
    """A dri_linearise result (and its flag bytes) against the oracle's
    linearisation `lin` and assembled system (H, b, cost) at the same state:
    per-pixel validity and ICP association bit-exact outside the margin pixels,
    counts equal to the kernel's own flags, every system within the bar (with
    the allowance of the margin pixels decided differently)."""
    gi, gr = (flags & 1) != 0, (flags & 2) != 0
    mi, mr = lin["icp_margin"], lin["rgb_margin"]
    bad_i = int((gi[~mi] != lin["icp_valid"][~mi]).sum())
    bad_r = int((gr[~mr] != lin["rgb_valid"][~mr]).sum())
    assert bad_i == 0, f"{what}: ICP validity differs at {bad_i} non-margin pixels"
    assert bad_r == 0, f"{what}: photometric validity differs at {bad_r} non-margin pixels"
    assert out.n_icp == gi.sum() and out.n_rgb == gr.sum()
    check_margins(out, flags, lin, what)
    al = margin_allowance(lin, flags, cur, ref, x0, x1, cfg)
    check_system(np.array(out.H_icp).reshape(6, 6), out.b_icp, lin["H_icp"], lin["b_icp"],
                 lin["cost_icp"], rel=rel, what=f"{what} ICP", allow=al["icp"])
    check_system(np.array(out.H_rgb).reshape(6, 6), out.b_rgb, lin["H_rgb"][6:, 6:], lin["b_rgb"][6:],
                 lin["cost_rgb"], rel=rel, what=f"{what} RGB", allow=al["rgb"])
    check_system(np.array(out.H).reshape(34, 34), out.b, H, b, cost, rel=rel, what=f"{what} joint",
                 allow=al["joint"])
    return al
