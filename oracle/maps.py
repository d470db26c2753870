"""Image pyramid, vertex / normal / intensity-gradient maps and reference maps.

Oracle code (test infrastructure only).  The paper minimises its cost "with a
three level coarse-to-fine pyramid scheme" (Sec. IV-D) and evaluates Eq. 3
(photometric) and Eq. 4 (point-to-plane ICP) on vertex, normal and intensity
maps, without describing how they are built.  Readings used here:

* Pyramid: level l halves level l-1 (floor of odd sizes).  Depth is the mean
  of the samples > 0 in each 2x2 block (0 if none); intensity is the plain
  2x2 mean.  Intrinsics scale as f_l = f / 2^l, c_l = (c + 0.5) / 2^l - 0.5.
  Every level is an FP32 map, as the level-0 images are: the depth mean adds
  the valid samples one at a time in FP32 in the block's row-major order and
  divides the sum by their count in FP32; the intensity mean is
  ((I00 + I01) + (I10 + I11)) / 4 in FP32.  (Each IEEE operation rounds to
  nearest even, so the level is defined to the bit; the normals and vertices
  built from it are then FP64 functions of the same stored values.)
* Vertex map: v = d K_l^-1 [u, v, 1]^T for depths in [depth_min, depth_max].
* Normal map: n = normalise((v(x+1,y) - v) x (v(x,y+1) - v)), flipped so that
  n . v < 0 (facing the camera); invalid on the last row / column, where a
  neighbour is invalid, or where the cross product vanishes.
* Intensity gradient: central differences (I(x+1) - I(x-1)) / 2 and
  (I(y+1) - I(y-1)) / 2; zero on the one-pixel border.
* Reference maps (the "global model" of Eq. 4, here the previous frame's maps
  moved into W with its final pose): V_W = R_ref v + r_ref, N_W = R_ref n,
  intensity and its gradient, and the pose T_ref they were made at.
* Uploaded reference (a model prediction rendered at T_ref, given as world-frame
  vertex and normal maps and an intensity image at level 0; the paper renders
  it from its surfel model, Sec. IV-B): a pixel has a surface where its normal
  is non-zero; its depth is the z of its vertex in the reference camera (the
  vertex of a prediction rendered from T_ref lies on its pixel's ray, and the
  maps keep that depth); its normal is kept where that depth is in range.
  Coarser levels: depth and intensity as for a live frame, the normal is the
  2x2 mean of the non-zero normals, renormalised (zero if none), kept where the
  level's depth is in range.
* Reduced-precision storage (cfg.fp16_maps): the camera-frame normals and the
  intensity gradients are rounded to IEEE half precision (round to nearest
  even) where they are stored, before any use; everything else stays FP64.
  This is the storage format of the FP16-map variant, so that variant can be
  compared with an oracle that sees the same maps.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def downsample_depth(d):
    """2x2 mean of the valid (> 0) samples; 0 where none is valid.  FP32 map:
    the finer level's stored (FP32) values are added one at a time in FP32 in
    the order (0, 0), (0, 1), (1, 0), (1, 1) of the block, and the sum is
    divided by the count in FP32."""
    d = np.asarray(d, dtype=np.float64).astype(np.float32)
    h, w = d.shape[0] // 2, d.shape[1] // 2
    s = np.zeros((h, w), dtype=np.float32)
    n = np.zeros((h, w), dtype=np.float32)
    for dy in (0, 1):
        for dx in (0, 1):
            v = d[dy: 2 * h: 2, dx: 2 * w: 2]
            ok = v > 0
            s = np.where(ok, s + v, s)
            n = n + ok.astype(np.float32)
    out = np.where(n > 0, s / np.maximum(n, np.float32(1)), np.float32(0))
    return out.astype(np.float64)


def downsample_intensity(img):
    """2x2 mean, FP32 map: ((I00 + I01) + (I10 + I11)) * 0.25 in FP32."""
    I = np.asarray(img, dtype=np.float64).astype(np.float32)
    h, w = I.shape[0] // 2, I.shape[1] // 2
    top = I[0: 2 * h: 2, 0: 2 * w: 2] + I[0: 2 * h: 2, 1: 2 * w: 2]
    bottom = I[1: 2 * h: 2, 0: 2 * w: 2] + I[1: 2 * h: 2, 1: 2 * w: 2]
    return ((top + bottom) * np.float32(0.25)).astype(np.float64)


def pyramid(depth, intensity, levels):
    ds = [np.asarray(depth, dtype=np.float64)]
    Is = [np.asarray(intensity, dtype=np.float64)]
    for _ in range(1, levels):
        ds.append(downsample_depth(ds[-1]))
        Is.append(downsample_intensity(Is[-1]))
    return ds, Is


def depth_valid(d, cfg):
    return (d >= cfg.depth_min) & (d <= cfg.depth_max)


def vertex_map(d, cam, cfg):
    """Back-projection rho(u, d) = d K^-1 [u, v, 1]^T (Eq. 3), camera frame."""
    h, w = d.shape
    u = np.arange(w, dtype=np.float64)[None, :]
    v = np.arange(h, dtype=np.float64)[:, None]
    V = np.stack(np.broadcast_arrays(d * (u - cam["cx"]) / cam["fx"],
                                     d * (v - cam["cy"]) / cam["fy"], d), axis=-1)
    valid = depth_valid(d, cfg)
    return V, valid


def normal_map(V, valid):
    """Normalised cross product of forward differences, facing the camera."""
    h, w, _ = V.shape
    N = np.zeros_like(V)
    ok = np.zeros((h, w), dtype=bool)
    dx = V[:-1, 1:] - V[:-1, :-1]
    dy = V[1:, :-1] - V[:-1, :-1]
    c = np.cross(dx, dy)
    nrm = np.linalg.norm(c, axis=-1)
    good = valid[:-1, :-1] & valid[:-1, 1:] & valid[1:, :-1] & (nrm > 0)
    n = c / np.where(nrm > 0, nrm, 1.0)[..., None]
    flip = np.sum(n * V[:-1, :-1], axis=-1) > 0
    n = np.where(flip[..., None], -n, n)
    N[:-1, :-1] = np.where(good[..., None], n, 0.0)
    ok[:-1, :-1] = good
    return N, ok


def gradient_map(img):
    img = np.asarray(img, dtype=np.float64)
    g = np.zeros(img.shape + (2,))
    g[1:-1, 1:-1, 0] = 0.5 * (img[1:-1, 2:] - img[1:-1, :-2])
    g[1:-1, 1:-1, 1] = 0.5 * (img[2:, 1:-1] - img[:-2, 1:-1])
    return g


@dataclass
class FrameLevel:
    """Maps of the live frame at one pyramid level (camera frame C1)."""
    cam: dict
    depth: np.ndarray
    V: np.ndarray
    V_valid: np.ndarray
    N: np.ndarray
    N_valid: np.ndarray
    I: np.ndarray


@dataclass
class RefLevel:
    """Reference maps at one level, vertices and normals in W (Eq. 4)."""
    cam: dict
    V_W: np.ndarray
    N_W: np.ndarray
    valid: np.ndarray        # vertex and normal both valid
    I: np.ndarray
    G: np.ndarray            # intensity gradient (gx, gy) per pixel
    depth: np.ndarray        # kept for the margin test of the association


def half(a):
    """Round to IEEE half precision (nearest even) and back to FP64."""
    return np.asarray(a, dtype=np.float64).astype(np.float16).astype(np.float64)


def frame_levels(depth, intensity, cfg):
    ds, Is = pyramid(depth, intensity, cfg.levels)
    fp16 = getattr(cfg, "fp16_maps", False)
    out = []
    for l in range(cfg.levels):
        cam = cfg.level_camera(l)
        V, vv = vertex_map(ds[l], cam, cfg)
        N, nv = normal_map(V, vv)
        if fp16:
            N = half(N)
        out.append(FrameLevel(cam=cam, depth=ds[l], V=V, V_valid=vv, N=N, N_valid=nv, I=Is[l]))
    return out


def reference_from_frame(levels, R_ref, r_ref, fp16=False):
    """The live frame's maps become the next reference, moved into W with T_ref."""
    out = []
    for fl in levels:
        V_W = fl.V @ R_ref.T + r_ref
        N_W = fl.N @ R_ref.T
        G = gradient_map(fl.I)
        if fp16:
            G = half(G)
        out.append(RefLevel(cam=fl.cam, V_W=V_W, N_W=N_W, valid=fl.V_valid & fl.N_valid,
                            I=fl.I, G=G, depth=fl.depth))
    return out


def downsample_normals(N):
    """2x2 mean of the non-zero normals, renormalised; zero where none is."""
    N = np.asarray(N, dtype=np.float64)
    h, w = N.shape[0] // 2, N.shape[1] // 2
    blk = N[: 2 * h, : 2 * w].reshape(h, 2, w, 2, 3)
    nz = np.linalg.norm(blk, axis=-1) > 0
    s = np.where(nz[..., None], blk, 0.0).sum(axis=(1, 3))
    n = np.linalg.norm(s, axis=-1)
    return np.where((n > 0)[..., None], s / np.where(n > 0, n, 1.0)[..., None], 0.0)


def reference_from_upload(V_W, N_W, intensity, R_ref, r_ref, cfg):
    """Reference levels from an uploaded prediction: V_W, N_W (H x W x 3, world
    frame), intensity (H x W) at level 0, rendered at T_ref = (R_ref, r_ref)."""
    V_W = np.asarray(V_W, dtype=np.float64)
    N_W = np.asarray(N_W, dtype=np.float64)
    V_c = (V_W - r_ref) @ R_ref            # R_ref^T (V_W - r_ref), row vectors
    N_c = N_W @ R_ref
    surf = np.linalg.norm(N_c, axis=-1) > 0
    d = np.where(surf, V_c[..., 2], 0.0)
    N = np.where((surf & depth_valid(d, cfg))[..., None], N_c, 0.0)
    I = np.asarray(intensity, dtype=np.float64)
    fp16 = getattr(cfg, "fp16_maps", False)
    out = []
    for l in range(cfg.levels):
        if l:
            d = downsample_depth(d)
            I = downsample_intensity(I)
            N = downsample_normals(N)
            N = np.where(depth_valid(d, cfg)[..., None], N, 0.0)
        cam = cfg.level_camera(l)
        V, vv = vertex_map(d, cam, cfg)
        Ns = half(N) if fp16 else N
        nv = np.linalg.norm(Ns, axis=-1) > 0
        G = gradient_map(I)
        if fp16:
            G = half(G)
        out.append(RefLevel(cam=cam, V_W=V @ R_ref.T + r_ref, N_W=Ns @ R_ref.T, valid=vv & nv,
                            I=I, G=G, depth=d))
    return out
