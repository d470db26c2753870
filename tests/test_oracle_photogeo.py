"""Pins of the oracle's photometric (Eq. 3) and ICP (Eq. 4) terms."""
import numpy as np
import pytest

from conftest import oracle_config
from oracle import maps, photogeo
from oracle.so3 import State, boxplus, exp_so3
from paper_2207_10940_gb300 import synth


def _setup(seq, cfg, x0=None, x1=None):
    x0 = State.from_dict(seq.gt[0]) if x0 is None else x0
    x1 = State.from_dict(seq.gt[1]) if x1 is None else x1
    L0 = maps.frame_levels(seq.depth[0], seq.intensity[0], cfg)
    L1 = maps.frame_levels(seq.depth[1], seq.intensity[1], cfg)
    ref = maps.reference_from_frame(L0, x0.R, x0.r)
    return x0, x1, L1, ref


def _perturb(x, k, h):
    d = np.zeros(17)
    d[k] = h
    return boxplus(x, d)


@pytest.fixture(scope="module")
def lin_setup(pair_small):
    cfg = oracle_config(pair_small)
    rng = np.random.default_rng(5)
    x0g = State.from_dict(pair_small.gt[0])
    x1g = State.from_dict(pair_small.gt[1])
    d0 = np.zeros(17)
    d0[:6] = rng.normal(size=6) * 2e-3
    d1 = np.zeros(17)
    d1[:6] = rng.normal(size=6) * 4e-3
    x0, x1, L1, ref = _setup(pair_small, cfg)
    return cfg, boxplus(x0g, d0), boxplus(x1g, d1), L1, ref, x0g


def test_icp_jacobian_matches_finite_differences(lin_setup):
    cfg, x0, x1, L1, ref, xr = lin_setup
    h = 1e-7
    base = photogeo.linearise(L1[0], ref[0], xr.R, xr.r, x0, x1, cfg)
    checked = 0
    for k in range(6):
        p = photogeo.linearise(L1[0], ref[0], xr.R, xr.r, x0, _perturb(x1, k, h), cfg)
        m = photogeo.linearise(L1[0], ref[0], xr.R, xr.r, x0, _perturb(x1, k, -h), cfg)
        same = (p["px"]["xi"] == m["px"]["xi"]) & (p["px"]["yi"] == m["px"]["yi"])
        mask = base["icp_valid"] & p["icp_valid"] & m["icp_valid"] & same
        fd = (p["px"]["e_icp"] - m["px"]["e_icp"]) / (2 * h)
        J = base["px"]["J_icp"][..., k]
        np.testing.assert_allclose(fd[mask], J[mask], rtol=1e-5, atol=1e-6)
        checked += mask.sum()
    assert checked > 1000
    # ICP does not depend on x_0
    p = photogeo.linearise(L1[0], ref[0], xr.R, xr.r, _perturb(x0, 4, 1e-3), x1, cfg)
    np.testing.assert_array_equal(p["px"]["e_icp"], base["px"]["e_icp"])


def test_photometric_jacobian_is_gradient_times_projection_derivative(lin_setup):
    """J_RGB = grad I_0(x, y)^T d(x, y)/d(pose) for both poses (chain rule of Eq. 3);
    the projection derivative is taken by central differences."""
    cfg, x0, x1, L1, ref, xr = lin_setup
    h = 1e-7
    base = photogeo.linearise(L1[0], ref[0], xr.R, xr.r, x0, x1, cfg)
    G = base["px"]["G0"]
    for which, col0 in (("x0", 0), ("x1", 6)):
        for k in range(6):
            if which == "x0":
                p = photogeo.linearise(L1[0], ref[0], xr.R, xr.r, _perturb(x0, k, h), x1, cfg)
                m = photogeo.linearise(L1[0], ref[0], xr.R, xr.r, _perturb(x0, k, -h), x1, cfg)
            else:
                p = photogeo.linearise(L1[0], ref[0], xr.R, xr.r, x0, _perturb(x1, k, h), cfg)
                m = photogeo.linearise(L1[0], ref[0], xr.R, xr.r, x0, _perturb(x1, k, -h), cfg)
            mask = base["rgb_valid"] & p["rgb_valid"] & m["rgb_valid"]
            dx = (p["px"]["xp"] - m["px"]["xp"]) / (2 * h)
            dy = (p["px"]["yp"] - m["px"]["yp"]) / (2 * h)
            want = G[..., 0] * dx + G[..., 1] * dy
            J = base["px"]["J_rgb"][..., col0 + k]
            scale = np.abs(G).sum(-1) * (np.abs(dx) + np.abs(dy)) + 1e-12
            assert np.max(np.abs(want - J)[mask] / scale[mask]) < 1e-5
            assert mask.sum() > 2000


def test_photometric_jacobian_exact_on_a_linear_ramp(pair_small):
    """With a reference intensity linear in the pixel coordinates, bilinear
    interpolation and the central-difference gradient are exact, so e_RGB's
    finite differences must equal J_RGB inside the image."""
    cfg = oracle_config(pair_small)
    x0, x1, L1, ref = _setup(pair_small, cfg)
    rl = ref[0]
    hh, ww = rl.I.shape
    u = np.arange(ww)[None, :]
    v = np.arange(hh)[:, None]
    rl.I = 0.2 + 0.004 * u + 0.003 * v + 0.0 * u * v
    rl.G = maps.gradient_map(rl.I)
    rng = np.random.default_rng(9)
    x1 = boxplus(x1, np.r_[rng.normal(size=6) * 3e-3, np.zeros(11)])
    h = 1e-7
    base = photogeo.linearise(L1[0], rl, x0.R, x0.r, x0, x1, cfg)
    inner = ((base["px"]["xp"] >= 1) & (base["px"]["xp"] < ww - 2)
             & (base["px"]["yp"] >= 1) & (base["px"]["yp"] < hh - 2))
    for k in range(6):
        for which in ("x0", "x1"):
            a = (_perturb(x0, k, h), x1) if which == "x0" else (x0, _perturb(x1, k, h))
            b = (_perturb(x0, k, -h), x1) if which == "x0" else (x0, _perturb(x1, k, -h))
            p = photogeo.linearise(L1[0], rl, x0.R, x0.r, *a, cfg)
            m = photogeo.linearise(L1[0], rl, x0.R, x0.r, *b, cfg)
            mask = base["rgb_valid"] & p["rgb_valid"] & m["rgb_valid"] & inner
            fd = (p["px"]["e_rgb"] - m["px"]["e_rgb"]) / (2 * h)
            J = base["px"]["J_rgb"][..., k + (0 if which == "x0" else 6)]
            np.testing.assert_allclose(fd[mask], J[mask], rtol=1e-5, atol=1e-7)


def test_icp_residual_vanishes_at_ground_truth_on_planes(small_cam):
    """Noise-free walls: point-to-plane error at the true pose is zero up to the
    FP32 rounding of the stored depths (<= 1e-6 m) except at wall corners."""
    seq = synth.frame_pair(seed=7, cam=small_cam, imu_noise=False, sigma_d=0, sigma_I=0,
                           spheres=False)
    cfg = oracle_config(seq)
    x0, x1, L1, ref = _setup(seq, cfg)
    lin = photogeo.linearise(L1[0], ref[0], x0.R, x0.r, x0, x1, cfg)
    e = np.abs(lin["px"]["e_icp"][lin["icp_valid"]])
    assert lin["n_icp"] > 0.6 * small_cam.width * small_cam.height
    assert np.mean(e < 1e-6) > 0.98


def test_photometric_residual_vanishes_for_identity_motion(pair_small):
    cfg = oracle_config(pair_small)
    x0 = State.from_dict(pair_small.gt[0])
    L0 = maps.frame_levels(pair_small.depth[0], pair_small.intensity[0], cfg)
    ref = maps.reference_from_frame(L0, x0.R, x0.r)
    for l in range(cfg.levels):
        lin = photogeo.linearise(L0[l], ref[l], x0.R, x0.r, x0, x0, cfg)
        e = lin["px"]["e_rgb"][lin["rgb_valid"]]
        assert lin["n_rgb"] > 0.8 * L0[l].depth.size
        assert np.max(np.abs(e)) < 1e-12
        # ICP too: every valid point associates with itself
        assert np.max(np.abs(lin["px"]["e_icp"][lin["icp_valid"]])) < 1e-12


def test_normal_equations_symmetric_psd(lin_setup):
    cfg, x0, x1, L1, ref, xr = lin_setup
    lin = photogeo.linearise(L1[0], ref[0], xr.R, xr.r, x0, x1, cfg)
    for H in (lin["H_icp"], lin["H_rgb"]):
        np.testing.assert_allclose(H, H.T, rtol=1e-14, atol=0)
        ev = np.linalg.eigvalsh(H)
        assert ev.min() >= -1e-12 * np.trace(H)
    # the RGB block is rank 6 in 12-D: its x_0 block is -M times its x_1 block
    assert np.linalg.matrix_rank(lin["H_rgb"], tol=1e-9 * np.trace(lin["H_rgb"])) == 6


# ---------------------------------------------------------------------------
# Brute force on 8x8 images: per-pixel loops written independently of the
# vectorised oracle, from Eq. 3-4 and the readings of the association.
# ---------------------------------------------------------------------------

def _bf_vertex(d, u, v, K, cfg):
    if not (cfg.depth_min <= d <= cfg.depth_max):
        return None
    fx, fy, cx, cy = K
    return np.array([d * (u - cx) / fx, d * (v - cy) / fy, d])


def _bf_normal(D, u, v, K, cfg):
    h, w = D.shape
    if u + 1 >= w or v + 1 >= h:
        return None
    p = _bf_vertex(D[v, u], u, v, K, cfg)
    px = _bf_vertex(D[v, u + 1], u + 1, v, K, cfg)
    py = _bf_vertex(D[v + 1, u], u, v + 1, K, cfg)
    if p is None or px is None or py is None:
        return None
    a, b = px - p, py - p
    n = np.array([a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]])
    L = np.sqrt(n @ n)
    if L == 0:
        return None
    n = n / L
    return -n if n @ p > 0 else n


def _bf_pixel_lookup(img, x, y):
    x0, y0 = int(np.floor(x)), int(np.floor(y))
    ax, ay = x - x0, y - y0
    return ((1 - ax) * (1 - ay) * img[y0][x0] + ax * (1 - ay) * img[y0][x0 + 1]
            + (1 - ax) * ay * img[y0 + 1][x0] + ax * ay * img[y0 + 1][x0 + 1])


def _bf_linearise(D1, I1, D0, I0, K, cfg, Rref, rref, R0, r0, R1, r1, occ_thr=0.0, dw=0):
    h, w = D1.shape
    fx, fy, cx, cy = K
    # reference gradient, border zero
    Gx = [[0.0] * w for _ in range(h)]
    Gy = [[0.0] * w for _ in range(h)]
    for y in range(1, h - 1):
        for x in range(1, w - 1):
            Gx[y][x] = (I0[y, x + 1] - I0[y, x - 1]) / 2.0
            Gy[y][x] = (I0[y + 1, x] - I0[y - 1, x]) / 2.0
    cos_thr = np.cos(np.deg2rad(cfg.icp_angle_thr_deg))
    Hi = np.zeros((6, 6))
    bi = np.zeros(6)
    ni = 0
    Hr = np.zeros((12, 12))
    br = np.zeros(12)
    nr = 0
    for v in range(h):
        for u in range(w):
            p = _bf_vertex(D1[v, u], u, v, K, cfg)
            if p is None:
                continue
            s1 = R1 @ p
            pw = s1 + r1
            # ICP
            n1 = _bf_normal(D1, u, v, K, cfg)
            if n1 is not None:
                q = Rref.T @ (pw - rref)
                if q[2] > 0:
                    xi = int(np.floor(fx * q[0] / q[2] + cx + 0.5))
                    yi = int(np.floor(fy * q[1] / q[2] + cy + 0.5))
                    if 0 <= xi < w and 0 <= yi < h:
                        vr = _bf_vertex(D0[yi, xi], xi, yi, K, cfg)
                        nrm = _bf_normal(D0, xi, yi, K, cfg)
                        if vr is not None and nrm is not None:
                            V = Rref @ vr + rref
                            N = Rref @ nrm
                            if np.linalg.norm(pw - V) < cfg.icp_dist_thr and (R1 @ n1) @ N > cos_thr:
                                e = N @ (pw - V)
                                J = np.r_[N, np.cross(s1, N)]
                                wz = 1.0 / D1[v, u] ** 4 if dw else 1.0
                                Hi += wz * np.outer(J, J)
                                bi -= wz * J * e
                                ni += 1
            # photometric
            q0 = R0.T @ (pw - r0)
            if q0[2] > 0:
                x = fx * q0[0] / q0[2] + cx
                y = fy * q0[1] / q0[2] + cy
                if 0 <= x < w - 1 and 0 <= y < h - 1:
                    if occ_thr > 0:             # depth consistency at the nearest pixel
                        dref = D0[int(np.floor(y + 0.5)), int(np.floor(x + 0.5))]
                        if dref > 0 and abs(q0[2] - dref) > occ_thr:
                            continue
                    e = _bf_pixel_lookup(I0, x, y) - I1[v, u]
                    gx = _bf_pixel_lookup(Gx, x, y)
                    gy = _bf_pixel_lookup(Gy, x, y)
                    Z = q0[2]
                    a = np.array([fx * gx / Z, fy * gy / Z,
                                  -(fx * gx * q0[0] + fy * gy * q0[1]) / (Z * Z)])
                    wv = R0 @ a
                    J = np.r_[-wv, -np.cross(pw - r0, wv), wv, np.cross(s1, wv)]
                    Hr += np.outer(J, J)
                    br -= J * e
                    nr += 1
    Wi, Wr = 1 / cfg.sigma_d ** 2, 1 / cfg.sigma_I ** 2
    return Wi * Hi, Wi * bi, ni, Wr * Hr, Wr * br, nr


@pytest.mark.parametrize("seed,occ,dw", [(11, 0.0, 0), (12, 0.0, 0), (13, 0.0, 0), (11, 0.004, 0),
                                         (12, 0.004, 0), (13, 0.0, 1)])
def test_brute_force_8x8(seed, occ, dw):
    cam = synth.Camera(8, 8, 8.0, 8.0, 4.0, 4.0)
    seq = synth.frame_pair(seed=seed, cam=cam, rot_deg=3.0, trans_m=0.05)
    cfg = oracle_config(seq, levels=1, iters=(1,), occlusion_thr=occ, icp_depth_weight=dw)
    rng = np.random.default_rng(seed)
    x0, x1, L1, ref = _setup(seq, cfg)
    xr = x0
    x0 = boxplus(x0, np.r_[rng.normal(size=6) * 1e-2, np.zeros(11)])
    x1 = boxplus(x1, np.r_[rng.normal(size=6) * 1e-2, np.zeros(11)])
    lin = photogeo.linearise(L1[0], ref[0], xr.R, xr.r, x0, x1, cfg)
    K = (cam.fx, cam.fy, cam.cx, cam.cy)
    D1 = seq.depth[1].astype(np.float64)
    D0 = seq.depth[0].astype(np.float64)
    Hi, bi, ni, Hr, br, nr = _bf_linearise(D1, seq.intensity[1].astype(np.float64), D0,
                                           seq.intensity[0].astype(np.float64), K, cfg,
                                           xr.R, xr.r, x0.R, x0.r, x1.R, x1.r, occ, dw)
    assert ni == lin["n_icp"] and nr == lin["n_rgb"]
    assert nr > 20 if occ == 0 else nr > 0
    if occ > 0:                        # the test rejects something on these scenes
        assert nr < photogeo.linearise(L1[0], ref[0], xr.R, xr.r, x0, x1,
                                       oracle_config(seq, levels=1, iters=(1,)))["n_rgb"]
    np.testing.assert_allclose(lin["H_icp"], Hi, rtol=1e-12, atol=1e-9 * max(1, np.abs(Hi).max()))
    np.testing.assert_allclose(lin["b_icp"], bi, rtol=1e-12, atol=1e-9 * max(1, np.abs(bi).max()))
    np.testing.assert_allclose(lin["H_rgb"], Hr, rtol=1e-12, atol=1e-9 * np.abs(Hr).max())
    np.testing.assert_allclose(lin["b_rgb"], br, rtol=1e-12, atol=1e-9 * np.abs(br).max())


def test_margin_flags_mark_near_threshold_pixels(pair_small):
    """A pixel moved onto a rounding boundary of the association is flagged."""
    cfg = oracle_config(pair_small)
    x0, x1, L1, ref = _setup(pair_small, cfg)
    lin = photogeo.linearise(L1[0], ref[0], x0.R, x0.r, x0, x1, cfg)
    assert lin["icp_margin"].sum() < 0.01 * lin["n_icp"] + 5
    # shift the reference camera so that x_ref + 0.5 of pixel column 40 is an integer
    cam = L1[0].cam
    xr = State.from_dict(pair_small.gt[0])
    q = xr.R.T @ (x1.R @ L1[0].V[30, 40] + x1.r - xr.r)
    x = cam["fx"] * q[0] / q[2] + cam["cx"] + 0.5
    shift = (np.round(x) - x + 3e-5) * q[2] / cam["fx"]
    r_ref = xr.r - xr.R @ np.array([shift, 0.0, 0.0])
    lin2 = photogeo.linearise(L1[0], ref[0], xr.R, r_ref, x0, x1, cfg)
    if L1[0].V_valid[30, 40] and L1[0].N_valid[30, 40]:
        assert lin2["icp_margin"][30, 40]


def test_rotation_of_reference_frame_leaves_icp_invariant(pair_small):
    """Moving the whole problem by a rigid transform of W changes nothing."""
    cfg = oracle_config(pair_small)
    x0, x1, L1, ref = _setup(pair_small, cfg)
    lin = photogeo.linearise(L1[0], ref[0], x0.R, x0.r, x0, x1, cfg)
    A = exp_so3([0.3, -0.2, 0.5])
    t = np.array([1.0, 2.0, -0.5])

    def move(x):
        y = x.copy()
        from oracle.so3 import rot_to_quat
        y.q = rot_to_quat(A @ x.R)
        y.r = A @ x.r + t
        return y

    y0, y1 = move(x0), move(x1)
    ref2 = maps.reference_from_frame(
        maps.frame_levels(pair_small.depth[0], pair_small.intensity[0], cfg), y0.R, y0.r)
    lin2 = photogeo.linearise(L1[0], ref2[0], y0.R, y0.r, y0, y1, cfg)
    assert lin2["n_icp"] == lin["n_icp"] and lin2["n_rgb"] == lin["n_rgb"]
    np.testing.assert_allclose(lin2["cost_icp"], lin["cost_icp"], rtol=1e-9)
    np.testing.assert_allclose(lin2["cost_rgb"], lin["cost_rgb"], rtol=1e-9)
