"""Pins of the oracle's pyramid and map construction (Sec. IV-D pyramid; Eq. 3-4 inputs)."""
import numpy as np

from oracle import maps
from oracle.params import TrackerConfig


def _cfg(w=16, h=12, f=14.0):
    return TrackerConfig(w, h, f, f, w / 2.0, h / 2.0, levels=3, iters=(1, 1, 1),
                         R_CS=np.eye(3), r_CS=np.zeros(3))


def test_depth_downsample_means_valid_samples():
    d = np.array([[1.0, 3.0, 0.0, 0.0],
                  [0.0, 2.0, 0.0, 5.0],
                  [1.0, 1.0, 2.0, 4.0],
                  [1.0, 1.0, 6.0, 0.0]])
    out = maps.downsample_depth(d)
    np.testing.assert_array_equal(out, [[2.0, 5.0], [1.0, 4.0]])
    assert maps.downsample_depth(np.zeros((4, 4))).sum() == 0.0


def test_depth_downsample_is_an_fp32_map_summed_in_block_order():
    """Each level is stored in FP32 and its mean is computed in FP32: within a
    few FP32 units of the exact mean; with one large and three tiny samples the
    row-major order (large one first) decides the bits, worked by hand in IEEE
    single precision: 1 + 2^-24 rounds to 1 (a tie, to even) three times, so
    the sum is 1 and the mean 0.25, where adding the tiny ones first would give
    (1 + 2^-22) / 4."""
    rng = np.random.default_rng(3)
    d = rng.uniform(0.3, 8.0, size=(64, 64)).astype(np.float32).astype(np.float64)
    d[rng.uniform(size=d.shape) < 0.2] = 0.0
    out = maps.downsample_depth(d)
    assert out.dtype == np.float64 and np.all(out.astype(np.float32) == out)   # FP32 values
    blk = d.reshape(32, 2, 32, 2)
    n = (blk > 0).sum(axis=(1, 3))
    exact = np.where(n > 0, blk.sum(axis=(1, 3)) / np.maximum(n, 1), 0.0)
    assert np.all(np.abs(out - exact) <= 4 * 2.0 ** -23 * exact)
    t = 2.0 ** -24
    assert maps.downsample_depth(np.array([[1.0, t], [t, t]]))[0, 0] == 0.25
    assert maps.downsample_depth(np.array([[t, t], [t, 1.0]]))[0, 0] == (1.0 + 2.0 ** -22) / 4
    # three valid samples: the FP32 quotient of the FP32 sum
    three = maps.downsample_depth(np.array([[0.0, 1.0], [1.0, 2.0 ** -23 + 1.0]]))[0, 0]
    assert three == float(np.float32(np.float32(3.0 + 2.0 ** -23) / np.float32(3.0)))


def test_intensity_downsample_is_block_mean_and_odd_sizes_floor():
    img = np.arange(35, dtype=np.float64).reshape(5, 7)
    out = maps.downsample_intensity(img)
    assert out.shape == (2, 3)
    np.testing.assert_allclose(out[0, 0], (0 + 1 + 7 + 8) / 4.0)
    np.testing.assert_allclose(out[1, 2], (18 + 19 + 25 + 26) / 4.0)


def test_level_intrinsics_match_block_centres():
    """A 3-D point seen at level-(l-1) pixel x sits at (x - 0.5) / 2 on level l."""
    cfg = _cfg(640, 480, 554.0)
    rng = np.random.default_rng(0)
    P = rng.uniform([-1, -1, 1], [1, 1, 3], size=(50, 3))
    for l in range(1, 3):
        a, b = cfg.level_camera(l - 1), cfg.level_camera(l)
        xa = a["fx"] * P[:, 0] / P[:, 2] + a["cx"]
        xb = b["fx"] * P[:, 0] / P[:, 2] + b["cx"]
        ya = a["fy"] * P[:, 1] / P[:, 2] + a["cy"]
        yb = b["fy"] * P[:, 1] / P[:, 2] + b["cy"]
        np.testing.assert_allclose(xb, (xa - 0.5) / 2.0, atol=1e-12)
        np.testing.assert_allclose(yb, (ya - 0.5) / 2.0, atol=1e-12)
        assert b["width"] == a["width"] // 2 and b["height"] == a["height"] // 2


def _plane_depth(cam, n, dist):
    """Exact z-depth of the plane n . X = dist seen by the camera."""
    u = np.arange(cam["width"], dtype=np.float64)[None, :]
    v = np.arange(cam["height"], dtype=np.float64)[:, None]
    rx = (u - cam["cx"]) / cam["fx"]
    ry = (v - cam["cy"]) / cam["fy"]
    return dist / (n[0] * rx + n[1] * ry + n[2])


def test_vertex_and_normal_of_a_tilted_plane():
    cfg = _cfg()
    cam = cfg.level_camera(0)
    n = np.array([0.2, -0.3, 1.0])
    n /= np.linalg.norm(n)
    d = _plane_depth(cam, n, 2.0)
    V, vv = maps.vertex_map(d, cam, cfg)
    assert vv.all()
    np.testing.assert_allclose(V @ n, 2.0, atol=1e-12)        # every vertex on the plane
    np.testing.assert_allclose(V[..., 2], d)
    N, nv = maps.normal_map(V, vv)
    assert nv[:-1, :-1].all() and not nv[-1].any() and not nv[:, -1].any()
    np.testing.assert_allclose(N[:-1, :-1], np.broadcast_to(-n, N[:-1, :-1].shape), atol=1e-12)


def test_normal_invalid_next_to_missing_depth_and_out_of_range():
    cfg = _cfg()
    cam = cfg.level_camera(0)
    d = np.full((12, 16), 2.0)
    d[5, 7] = 0.0
    d[2, 2] = 9.0               # beyond depth_max = 8
    V, vv = maps.vertex_map(d, cam, cfg)
    N, nv = maps.normal_map(V, vv)
    assert not vv[5, 7] and not vv[2, 2]
    for (y, x) in [(5, 7), (5, 6), (4, 7), (2, 2), (2, 1), (1, 2)]:
        assert not nv[y, x]
    assert nv[6, 8] and nv[0, 0]


def test_gradient_of_a_ramp_is_exact_inside_and_zero_on_border():
    u = np.arange(16, dtype=np.float64)[None, :]
    v = np.arange(12, dtype=np.float64)[:, None]
    img = 0.1 + 0.02 * u - 0.03 * v + 0 * u * v
    G = maps.gradient_map(img)
    np.testing.assert_allclose(G[1:-1, 1:-1, 0], 0.02, atol=1e-15)
    np.testing.assert_allclose(G[1:-1, 1:-1, 1], -0.03, atol=1e-15)
    assert np.all(G[0] == 0) and np.all(G[-1] == 0) and np.all(G[:, 0] == 0) and np.all(G[:, -1] == 0)


def test_reference_maps_are_moved_into_world():
    cfg = _cfg()
    rng = np.random.default_rng(3)
    d = rng.uniform(1.0, 3.0, (12, 16))
    I = rng.uniform(0, 1, (12, 16))
    lv = maps.frame_levels(d, I, cfg)
    from oracle.so3 import exp_so3
    R = exp_so3([0.1, -0.2, 0.3])
    r = np.array([0.5, -1.0, 2.0])
    ref = maps.reference_from_frame(lv, R, r)
    for fl, rl in zip(lv, ref):
        np.testing.assert_allclose(rl.V_W, fl.V @ R.T + r, atol=1e-14)
        np.testing.assert_allclose(np.linalg.norm(rl.N_W[rl.valid], axis=-1), 1.0, atol=1e-14)
        np.testing.assert_allclose((rl.N_W @ R)[rl.valid], fl.N[rl.valid], atol=1e-14)


def test_fp16_map_storage_rounds_normals_and_gradients_to_half(pair_small):
    """With fp16_maps the stored normals and gradients are exactly the IEEE
    half-precision roundings of the FP64 maps (relative error <= 2^-11 for
    normal-range values, as for any round-to-nearest binary16), the depth,
    vertices and intensities are untouched."""
    from oracle.params import TrackerConfig
    seq = pair_small
    cam = seq.cam
    exact = TrackerConfig(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, levels=2)
    half = TrackerConfig(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, levels=2, fp16_maps=True)
    le = maps.frame_levels(seq.depth[0], seq.intensity[0], exact)
    lh = maps.frame_levels(seq.depth[0], seq.intensity[0], half)
    for a, b in zip(le, lh):
        np.testing.assert_array_equal(b.N, a.N.astype(np.float16).astype(np.float64))
        np.testing.assert_array_equal(b.V, a.V)
        np.testing.assert_array_equal(b.I, a.I)
        big = np.abs(a.N) >= 2.0 ** -14
        assert np.all(np.abs(b.N - a.N)[big] <= 2.0 ** -11 * np.abs(a.N)[big])
        assert np.any(b.N != a.N)                      # rounding did happen
    R, r = np.eye(3), np.zeros(3)
    re = maps.reference_from_frame(le, R, r)
    rh = maps.reference_from_frame(lh, R, r, fp16=True)
    for a, b in zip(re, rh):
        np.testing.assert_array_equal(b.G, a.G.astype(np.float16).astype(np.float64))
        np.testing.assert_array_equal(b.I, a.I)


def _world_maps(level, R, r):
    return level.V @ R.T + r, np.where(level.N_valid[..., None], level.N, 0.0) @ R.T


def test_uploaded_reference_round_trip_at_level_zero(pair_small):
    """A frame's own level-0 maps moved into W and uploaded give back its depth
    and normals wherever it has a normal, and no surface elsewhere."""
    from oracle.params import TrackerConfig
    from oracle.so3 import exp_so3
    seq = pair_small
    cam = seq.cam
    cfg = TrackerConfig(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, levels=3)
    lv = maps.frame_levels(seq.depth[0], seq.intensity[0], cfg)
    R, r = exp_so3(np.array([0.3, -0.2, 0.5])), np.array([0.4, -1.0, 2.0])
    V_W, N_W = _world_maps(lv[0], R, r)
    ref = maps.reference_from_upload(V_W, N_W, lv[0].I, R, r, cfg)
    ok = lv[0].N_valid
    np.testing.assert_allclose(ref[0].depth[ok], lv[0].depth[ok], rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(ref[0].depth[~ok], 0.0)
    np.testing.assert_allclose((ref[0].N_W @ R)[ok], lv[0].N[ok], atol=1e-12)
    np.testing.assert_array_equal(ref[0].valid, ok)
    np.testing.assert_array_equal(ref[0].I, lv[0].I)
    for l in (1, 2):
        n = np.linalg.norm(ref[l].N_W, axis=-1)
        assert np.all((np.abs(n - 1.0) < 1e-12) | (n == 0))    # unit or none
        assert ref[l].depth.shape == lv[l].depth.shape


def test_uploaded_plane_keeps_its_normal_on_every_level():
    """Averaging identical unit normals gives that normal back: a fronto-parallel
    plane uploaded at any pose has the plane's normal at every level."""
    from oracle.params import TrackerConfig
    from oracle.so3 import exp_so3
    cfg = TrackerConfig(64, 48, 60.0, 60.0, 32.0, 24.0, levels=3)
    R, r = exp_so3(np.array([-0.1, 0.4, 0.2])), np.array([1.0, 2.0, -0.5])
    h, w = 48, 48 * 0 + 64
    u, v = np.meshgrid(np.arange(w), np.arange(h))
    d = np.full((h, w), 2.0)
    Vc = np.stack([d * (u - 32.0) / 60.0, d * (v - 24.0) / 60.0, d], axis=-1)
    Nc = np.broadcast_to(np.array([0.0, 0.0, -1.0]), (h, w, 3))
    ref = maps.reference_from_upload(Vc @ R.T + r, Nc @ R.T, np.full((h, w), 0.5), R, r, cfg)
    for lev in ref:
        np.testing.assert_allclose(lev.N_W @ R, np.broadcast_to([0.0, 0.0, -1.0], lev.N_W.shape),
                                   atol=1e-13)
        np.testing.assert_allclose(lev.depth, 2.0, rtol=1e-13)
        assert lev.valid.all()
