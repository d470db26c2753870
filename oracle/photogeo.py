"""Photometric (Eq. 3) and point-to-plane ICP (Eq. 4) terms at one pyramid level.

Oracle code (test infrastructure only).  For every live pixel u with a valid
depth it evaluates, in FP64 and in world coordinates:

ICP (Eq. 4, Sec. IV-B).  p_W = R_1 p + r_1 with p = rho(u, d).  Reading of the
"corresponding point in the global model": projective association into the
reference view at the fixed pose T_ref the reference was made at, nearest
pixel floor(x + 0.5), accepted when inside the image, the reference vertex and
normal are valid, ||p_W - V_W|| < d_thr and angle(R_1 n, N_W) < theta_thr.
  e_ICP = N_W . (p_W - V_W)
  de/d(dr_1, da_1) = [N_W ; s_1 x N_W],  s_1 = R_1 p          (left perturbation)
The ICP term depends on x_1 only.

Photometric (Eq. 3, Sec. IV-B).  p_0 = R_0^T (p_W - r_0) with the current
iterate of x_0, (x, y) = pi(K p_0); valid when z_0 > 0 and
(x, y) in [0, W-1) x [0, H-1) so the bilinear support is inside the image.
  e_RGB = I_0(x, y) - I_1(u)          (I_0, grad I_0 bilinear)
  a = (d pi / d p_0)^T grad I_0(x, y),   w = R_0 a
  de/d(dr_1, da_1) = [w ; s_1 x w]
  de/d(dr_0, da_0) = -[w ; (p_W - r_0) x w]
Both Jacobians follow from the left perturbations of Eq. 2 and are pinned
against central finite differences by the CPU tests.

Weights are the constant inverse covariances W_ICP = 1/sigma_d^2 and
W_RGB = 1/sigma_I^2 (Eq. 6).  Returned systems follow Eq. 7's H dx = b with
H = sum W J J^T and b = -sum W J e.

Margin pixels.  A pixel whose accept / reject decision sits within 1e-4 px of
an image bound or rounding boundary, or within a relative 1e-5 of a metric
threshold (depth range, z > 0, distance, normal angle, normal orientation), is
flagged: an FP32 implementation may legitimately decide it the other way, so
exact count comparisons exclude these pixels and count them separately.  With
normals stored in FP16 (cfg.fp16_maps) the angle test's margin is 4 * 2^-11 in
cos: the stored normal is a rounding, and rounding an FP32-computed normal may
give the neighbouring half-precision value of the FP64-computed one.
"""
from __future__ import annotations

import numpy as np

from .maps import FrameLevel, RefLevel, depth_valid

PX_MARGIN = 1e-4
REL_MARGIN = 1e-5
FP16_COS_MARGIN = 4.0 * 2.0 ** -11      # angle-test margin when normals are stored in FP16


def _near_rel(a, thr):
    return np.abs(a - thr) <= REL_MARGIN * abs(thr)


def _depth_margin(d, cfg):
    return _near_rel(d, cfg.depth_min) | _near_rel(d, cfg.depth_max)


def _shift(a, dy, dx, fill):
    """a[y+dy, x+dx] with `fill` outside."""
    out = np.full_like(a, fill)
    h, w = a.shape[:2]
    out[: h - dy, : w - dx] = a[dy:, dx:]
    return out


def _normal_margin(depth, V, N, cfg):
    """Decision margins of a normal: depth-range tests of the three depths it
    reads and the orientation test n . v < 0."""
    m = _depth_margin(depth, cfg) | _depth_margin(_shift(depth, 0, 1, 0.0), cfg) \
        | _depth_margin(_shift(depth, 1, 0, 0.0), cfg)
    vn = np.linalg.norm(V, axis=-1)
    nv = np.sum(N * V, axis=-1)
    m |= (np.linalg.norm(N, axis=-1) > 0) & (np.abs(nv) <= REL_MARGIN * np.maximum(vn, 1e-30))
    return m


def _bilinear(img, x, y):
    x0 = np.floor(x).astype(np.int64)
    y0 = np.floor(y).astype(np.int64)
    ax = x - x0
    ay = y - y0
    if img.ndim == 3:
        ax = ax[..., None]
        ay = ay[..., None]
    return ((1 - ax) * (1 - ay) * img[y0, x0] + ax * (1 - ay) * img[y0, x0 + 1]
            + (1 - ax) * ay * img[y0 + 1, x0] + ax * ay * img[y0 + 1, x0 + 1])


def linearise(cur: FrameLevel, ref: RefLevel, R_ref, r_ref, x0, x1, cfg):
    """Weighted normal equations of the ICP and photometric terms at (x0, x1)."""
    h, w = cur.depth.shape
    cam = cur.cam
    fx, fy, cx, cy = cam["fx"], cam["fy"], cam["cx"], cam["cy"]
    rw, rh = ref.cam["width"], ref.cam["height"]
    R0, r0, R1, r1 = x0.R, x0.r, x1.R, x1.r
    dv = depth_valid(cur.depth, cfg)
    p = cur.V
    s1 = p @ R1.T
    pW = s1 + r1

    # ---------------- ICP (Eq. 4) ----------------
    pr = (pW - r_ref) @ R_ref            # R_ref^T (p_W - r_ref)
    z = pr[..., 2]
    zpos = z > 0
    zs = np.where(zpos, z, 1.0)
    xr = fx * pr[..., 0] / zs + cx
    yr = fy * pr[..., 1] / zs + cy
    xi = np.floor(xr + 0.5)
    yi = np.floor(yr + 0.5)
    inb = zpos & (xi >= 0) & (xi <= rw - 1) & (yi >= 0) & (yi <= rh - 1)
    xc = np.clip(xi, 0, rw - 1).astype(np.int64)
    yc = np.clip(yi, 0, rh - 1).astype(np.int64)
    Vr = ref.V_W[yc, xc]
    Nr = ref.N_W[yc, xc]
    rvalid = inb & ref.valid[yc, xc]
    diff = pW - Vr
    dist = np.linalg.norm(diff, axis=-1)
    n1W = cur.N @ R1.T
    cosang = np.sum(n1W * Nr, axis=-1)
    cos_thr = np.cos(np.deg2rad(cfg.icp_angle_thr_deg))
    icp_valid = dv & cur.N_valid & rvalid & (dist < cfg.icp_dist_thr) & (cosang > cos_thr)
    e_icp = np.sum(Nr * diff, axis=-1)
    J_icp = np.concatenate([Nr, np.cross(s1, Nr)], axis=-1)

    cand = dv & cur.N_valid
    # margins of the decisions made per pixel in the linearisation itself (the
    # pixel's own depth range, z > 0, the rounding, distance and angle tests) ...
    m_icp_px = _depth_margin(cur.depth, cfg) & dv
    m_icp_px |= cand & (np.abs(z) <= REL_MARGIN * np.linalg.norm(pr, axis=-1))
    rx = xr + 0.5
    ry = yr + 0.5
    m_icp_px |= cand & zpos & ((np.abs(rx - np.round(rx)) < PX_MARGIN) |
                               (np.abs(ry - np.round(ry)) < PX_MARGIN))
    m_icp_px |= cand & rvalid & (_near_rel(dist, cfg.icp_dist_thr) | _near_rel(cosang, cos_thr))
    if getattr(cfg, "fp16_maps", False):
        # normals stored in half precision: an implementation that rounds a normal
        # computed in FP32 may land one half-precision unit (2^-11 relative) away
        # from the rounding of the FP64 normal, which moves cos by up to ~2 * 2^-11
        m_icp_px |= cand & rvalid & (np.abs(cosang - cos_thr) <= FP16_COS_MARGIN)
    # ... and of those made while the normal maps were built (the live pixel's
    # and the associated reference pixel's)
    ref_nm = _normal_margin(ref.depth, (ref.V_W - r_ref) @ R_ref, ref.N_W @ R_ref, cfg)
    m_icp = m_icp_px | (_normal_margin(cur.depth, cur.V, cur.N, cfg) & dv) | (cand & inb & ref_nm[yc, xc])

    # ---------------- photometric (Eq. 3) ----------------
    p0 = (pW - r0) @ R0                  # R_0^T (p_W - r_0)
    z0 = p0[..., 2]
    z0pos = z0 > 0
    z0s = np.where(z0pos, z0, 1.0)
    X0, Y0 = p0[..., 0], p0[..., 1]
    xp = fx * X0 / z0s + cx
    yp = fy * Y0 / z0s + cy
    rgb_valid = dv & z0pos & (xp >= 0) & (xp < rw - 1) & (yp >= 0) & (yp < rh - 1)
    # depth consistency (occlusion) test, when enabled: the point's depth in x_0's
    # camera against the reference depth at the nearest reference pixel
    occ_thr = getattr(cfg, "occlusion_thr", 0.0)
    if occ_thr > 0:
        xn = np.clip(np.floor(np.where(rgb_valid, xp, 0.0) + 0.5), 0, rw - 1).astype(np.int64)
        yn = np.clip(np.floor(np.where(rgb_valid, yp, 0.0) + 0.5), 0, rh - 1).astype(np.int64)
        dref = ref.depth[yn, xn]
        occ_gap = np.abs(z0 - dref)
        inside = rgb_valid.copy()
        rgb_valid &= ~((dref > 0) & (occ_gap > occ_thr))
    xs = np.where(rgb_valid, xp, 0.0)
    ys = np.where(rgb_valid, yp, 0.0)
    I0 = _bilinear(ref.I, xs, ys)
    G0 = _bilinear(ref.G, xs, ys)
    e_rgb = I0 - cur.I
    gx, gy = G0[..., 0], G0[..., 1]
    a = np.stack([fx * gx / z0s, fy * gy / z0s,
                  -(fx * gx * X0 + fy * gy * Y0) / (z0s * z0s)], axis=-1)
    wv = a @ R0.T                        # R_0 a
    J1 = np.concatenate([wv, np.cross(s1, wv)], axis=-1)
    J0 = -np.concatenate([wv, np.cross(pW - r0, wv)], axis=-1)
    J_rgb = np.concatenate([J0, J1], axis=-1)

    m_rgb = _depth_margin(cur.depth, cfg) & dv
    m_rgb |= dv & (np.abs(z0) <= REL_MARGIN * np.linalg.norm(p0, axis=-1))
    m_rgb |= dv & z0pos & ((np.abs(xp) <= PX_MARGIN) | (np.abs(xp - (rw - 1)) <= PX_MARGIN) |
                           (np.abs(yp) <= PX_MARGIN) | (np.abs(yp - (rh - 1)) <= PX_MARGIN))
    if occ_thr > 0:
        # the nearest reference pixel's rounding and the depth gap's threshold
        fxn, fyn = xp + 0.5, yp + 0.5
        m_rgb |= inside & ((np.abs(fxn - np.round(fxn)) < PX_MARGIN) |
                           (np.abs(fyn - np.round(fyn)) < PX_MARGIN))
        m_rgb |= inside & (dref > 0) & _near_rel(occ_gap, occ_thr)

    W_icp = 1.0 / cfg.sigma_d ** 2
    W_rgb = 1.0 / cfg.sigma_I ** 2
    Ji, ei = J_icp[icp_valid], e_icp[icp_valid]
    if getattr(cfg, "icp_depth_weight", 0):
        # per-pixel weight 1 / z^4 (sigma_d(z) = sigma_d z^2): scale J and e by 1 / z^2
        sw = 1.0 / cur.depth[icp_valid].astype(np.float64) ** 2
        Ji, ei = Ji * sw[:, None], ei * sw
    Jr, er = J_rgb[rgb_valid], e_rgb[rgb_valid]
    return dict(
        H_icp=W_icp * Ji.T @ Ji, b_icp=-W_icp * Ji.T @ ei, cost_icp=W_icp * float(ei @ ei),
        n_icp=int(icp_valid.sum()),
        H_rgb=W_rgb * Jr.T @ Jr, b_rgb=-W_rgb * Jr.T @ er, cost_rgb=W_rgb * float(er @ er),
        n_rgb=int(rgb_valid.sum()),
        icp_valid=icp_valid, rgb_valid=rgb_valid, icp_margin=m_icp, rgb_margin=m_rgb,
        # the photometric margins are all decided per pixel in the linearisation
        icp_margin_px=m_icp_px, rgb_margin_px=m_rgb,
        # per-pixel values (also where invalid) for finite-difference checks
        px=dict(e_icp=e_icp, J_icp=J_icp, e_rgb=e_rgb, J_rgb=J_rgb, xi=xi, yi=yi, xp=xp, yp=yp,
                G0=G0),
    )

