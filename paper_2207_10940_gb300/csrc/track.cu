// Fused per-pixel Gauss-Newton linearisation of the photometric (Eq. 3) and
// point-to-plane ICP (Eq. 4) terms at one pyramid level, block-reduced into the
// normal equations of Eq. 7 (Sec. IV-B, IV-D).
//
// A thread evaluates one term only and carries that term's 29 sums: half the
// registers of a thread that does both, more warps resident per SM to hide the
// latency of the dependent gathers.  Batched kernel: a block of 8 warps takes
// one term over a tile of 32 columns x 8 * ppt rows (warp w: rows w, w + 8, ...),
// the two terms of a tile being neighbouring blocks, so a block never waits at
// its final barrier for the other (slower) term.  By-value kernel (parity,
// per-pixel flags): warps 0-3 ICP and 4-7 photometric over the same 32 x 4 * ppt
// pixels, so the two validity bits of a pixel meet in shared memory.  Each
// gather is one vector load of a per-pixel pack (packs.cuh): the ICP term reads
// pack A (normal + depth) of the live pixel and of the associated reference
// pixel, the photometric term the live depth and intensity and four pack-B taps
// (intensity + gradient) of the reference.  Each thread loads its next row's
// live samples before it works on the current one.  Per pixel, in FP32:
//
//   p   = d K^-1 [u, v, 1]^T                       live point, camera frame C1
//   ICP: D = A_ref p + t_ref  with A_ref = R_ref^T R_1 - I, t_ref = R_ref^T (r_1 - r_ref),
//        so p_ref = p + D is the point in the reference camera; the projection is
//        x = u + f (D_x - r_x D_z) / z  (the identity warp plus a small displacement
//        kept separate from the integer u, so neither cancels nor rounds at large
//        image coordinates), nearest pixel u + floor(disp + 0.5), reference vertex
//        V = d_ref K^-1 [x_i, y_i, 1]^T and normal N (reference camera frame),
//        accepted when ||p_ref - V|| < d_thr and (R_rel n) . N > cos(theta_thr);
//        e = N . ((p - V) + D),  J_loc = [N ; (p + A_ref p) x N].
//   RGB: the same with A_0 = R_0^T R_1 - I, t_0 = R_0^T (r_1 - r_0); valid when z_0 > 0
//        and (x, y) in [0, W-1) x [0, H-1); e = I_0(x, y) - I_1(u) (bilinear),
//        g = bilinear grad I_0,  a = (f_x g_x / z, f_y g_y / z, -(g_x (x - c_x) + g_y (y - c_y)) / z),
//        J_loc = [a ; (p + A_0 p) x a].
//
// The local Jacobians are the world-frame ones of Eq. 3-4 rotated by
// diag(R^T, R^T) (R = R_ref or R_0); the solver rotates the reduced 6x6 systems
// back in FP64.  Each thread accumulates its term's 29 values (upper J J^T, J e,
// e^2, count) in FP32; a warp transposes and sums them with 31 shuffles, the
// block adds its warps per term in fixed order into one FP64 (or FP32)
// partial of 58 values; the partials are folded in two fixed-order levels
// (groups of blocks, then the groups) into ctrl->sums: deterministic, no float
// atomics.
#include <cuda_fp16.h>

#include "dri_internal.h"
#include "packs.cuh"

namespace dri {

namespace {

__device__ __forceinline__ void accumulate(float* a, const float* J, float e) {
  int k = 0;
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = i; j < 6; ++j) {
      a[k] = fmaf(J[i], J[j], a[k]);
      ++k;
    }
#pragma unroll
  for (int i = 0; i < 6; ++i) a[21 + i] = fmaf(J[i], e, a[21 + i]);
  a[27] = fmaf(e, e, a[27]);
  a[28] += 1.f;
}

// Rows ahead of the current one whose live and reference samples (at the same
// pixel) each thread asks L2 to fetch: the gathers of a later row then find
// their lines in L2 instead of waiting on HBM (0: none).
constexpr int kPrefetchRows = 4;

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Live-frame samples of one pixel: depth and the term's own map (the normal for
// ICP, the intensity for the photometric term).
struct Live {
  float d, a, b, c;
};

// ICP term (Eq. 4) of the pixel (u, v) with live depth d and normal n1.  *assoc
// receives the associated reference pixel of an accepted correspondence as
// (x_i mod 4) | (y_i mod 4) << 2 (parity output; unused otherwise).
template <typename T, bool DW>
__device__ __forceinline__ bool icp_pixel(const TrackParams& p, const LevelGeom& g, const float* A,
                                          const float* t, const void* __restrict__ A0,
                                          const float* __restrict__ D0, int u, int v, const Live& L,
                                          float* acc, unsigned* assoc) {
  const float n1x = L.a, n1y = L.b, n1z = L.c;
  if (n1x == 0.f && n1y == 0.f && n1z == 0.f) return false;
  const float d = L.d;
  const float rx = ((float)u - g.cx) * g.ifx;
  const float ry = ((float)v - g.cy) * g.ify;
  const float px = d * rx, py = d * ry, pz = d;
  const float ex = fmaf(A[0], px, fmaf(A[1], py, fmaf(A[2], pz, t[0])));
  const float ey = fmaf(A[3], px, fmaf(A[4], py, fmaf(A[5], pz, t[1])));
  const float ez = fmaf(A[6], px, fmaf(A[7], py, fmaf(A[8], pz, t[2])));
  const float z = d + ez;
  if (!(z > 0.f)) return false;
  const float iz = __fdividef(1.f, z);
  const float sxp = g.fx * (fmaf(-rx, ez, ex) * iz);
  const float syp = g.fy * (fmaf(-ry, ez, ey) * iz);
  const bool sane = fabsf(sxp) < 1e7f && fabsf(syp) < 1e7f;   // int conversion in range
  const int xi = sane ? u + (int)floorf(sxp + 0.5f) : -1;
  const int yi = sane ? v + (int)floorf(syp + 0.5f) : -1;
  if (xi < 0 || xi >= g.w || yi < 0 || yi >= g.h) return false;
  const float4 n0 = Packs<T>::load_a(A0, D0, yi * g.w + xi);   // N (x, y, z), reference depth
  const float Nx = n0.x, Ny = n0.y, Nz = n0.z, dr = n0.w;
  if (Nx == 0.f && Ny == 0.f && Nz == 0.f) return false;
  const float Vx = dr * (((float)xi - g.cx) * g.ifx), Vy = dr * (((float)yi - g.cy) * g.ify);
  const float dx = (px - Vx) + ex, dy = (py - Vy) + ey, dz = (pz - dr) + ez;
  const float dist2 = dx * dx + dy * dy + dz * dz;
  const float mx = n1x + (A[0] * n1x + A[1] * n1y + A[2] * n1z);
  const float my = n1y + (A[3] * n1x + A[4] * n1y + A[5] * n1z);
  const float mz = n1z + (A[6] * n1x + A[7] * n1y + A[8] * n1z);
  const float cosang = mx * Nx + my * Ny + mz * Nz;
  if (!(dist2 < p.icp_dist2 && cosang > p.icp_cos)) return false;
  *assoc = (unsigned)(xi & 3) | ((unsigned)(yi & 3) << 2);
  const float e = Nx * dx + Ny * dy + Nz * dz;
  const float sx = px + (ex - t[0]), sy = py + (ey - t[1]), sz = pz + (ez - t[2]);
  const float J[6] = {Nx, Ny, Nz, sy * Nz - sz * Ny, sz * Nx - sx * Nz, sx * Ny - sy * Nx};
  if (DW) {                      // weight 1 / d^4 (sigma_d(d) = sigma_d d^2): J, e scaled by 1 / d^2
    const float w = __fdividef(1.f, d * d);
    const float Jw[6] = {J[0] * w, J[1] * w, J[2] * w, J[3] * w, J[4] * w, J[5] * w};
    accumulate(acc, Jw, e * w);
    return true;
  }
  accumulate(acc, J, e);
  return true;
}

// Photometric term (Eq. 3) of the pixel (u, v) with live depth d and intensity i1.
template <typename T, bool OCC>
__device__ __forceinline__ bool rgb_pixel(const LevelGeom& g, const float* A, const float* t,
                                          const void* __restrict__ B0, const float* __restrict__ D0,
                                          float occ_thr, int u, int v, const Live& L, float* acc) {
  const float d = L.d;
  const float rx = ((float)u - g.cx) * g.ifx;
  const float ry = ((float)v - g.cy) * g.ify;
  const float px = d * rx, py = d * ry, pz = d;
  const float ex = fmaf(A[0], px, fmaf(A[1], py, fmaf(A[2], pz, t[0])));
  const float ey = fmaf(A[3], px, fmaf(A[4], py, fmaf(A[5], pz, t[1])));
  const float ez = fmaf(A[6], px, fmaf(A[7], py, fmaf(A[8], pz, t[2])));
  const float z = d + ez;
  if (!(z > 0.f)) return false;
  const float iz = __fdividef(1.f, z);
  // displacement of the projection from (u, v): small, so FP32 keeps it to
  // ~1e-6 px, and integer parts of the position stay exact
  const float sxp = g.fx * (fmaf(-rx, ez, ex) * iz);
  const float syp = g.fy * (fmaf(-ry, ez, ey) * iz);
  const float fxp = floorf(sxp), fyp = floorf(syp);
  const bool sane = fabsf(sxp) < 1e7f && fabsf(syp) < 1e7f;   // int conversion in range
  const int xb = sane ? u + (int)fxp : -1, yb = sane ? v + (int)fyp : -1;
  if (xb < 0 || xb >= g.w - 1 || yb < 0 || yb >= g.h - 1) return false;
  const float ax = sxp - fxp, ay = syp - fyp;
  const int q = yb * g.w + xb;
  const float4 s00 = Packs<T>::load_b(B0, q), s01 = Packs<T>::load_b(B0, q + 1);
  const float4 s10 = Packs<T>::load_b(B0, q + g.w), s11 = Packs<T>::load_b(B0, q + g.w + 1);
  if (OCC) {                     // depth consistency at the nearest reference pixel
    const bool right = floorf(sxp + 0.5f) != fxp, down = floorf(syp + 0.5f) != fyp;
    const float dr = Packs<T>::kDepthInB
                         ? (down ? (right ? s11.w : s10.w) : (right ? s01.w : s00.w))
                         : __ldg(D0 + (yb + (down ? 1 : 0)) * g.w + xb + (right ? 1 : 0));
    if (dr > 0.f && fabsf(z - dr) > occ_thr) return false;
  }
  const float w00 = (1.f - ax) * (1.f - ay), w01 = ax * (1.f - ay);
  const float w10 = (1.f - ax) * ay, w11 = ax * ay;
  const float iv = w00 * s00.x + w01 * s01.x + w10 * s10.x + w11 * s11.x;
  const float gx = w00 * s00.y + w01 * s01.y + w10 * s10.y + w11 * s11.y;
  const float gy = w00 * s00.z + w01 * s01.z + w10 * s10.z + w11 * s11.z;
  const float e = iv - L.a;
  const float a0 = g.fx * gx * iz, a1 = g.fy * gy * iz;
  const float a2 = -(gx * (((float)u - g.cx) + sxp) + gy * (((float)v - g.cy) + syp)) * iz;
  const float sx = px + (ex - t[0]), sy = py + (ey - t[1]), sz = pz + (ez - t[2]);
  const float J[6] = {a0, a1, a2, sy * a2 - sz * a1, sz * a0 - sx * a2, sx * a1 - sy * a0};
  accumulate(acc, J, e);
  return true;
}

// One tile of one image (single-term: 32 x 8 * ppt pixels of `term`; mixed:
// 32 x 4 * ppt pixels, both terms): (bx, by) its tile
// coordinates, bid its index in the image's fold order.
// Optional terms, compile-time variants of the pixel kernels (OPT bits): the
// photometric occlusion test and the depth-dependent ICP weight.
constexpr int kOptOcc = 1, kOptDepthWeight = 2;

template <typename T, typename P, bool FLAGS, bool SPLIT, int OPT>
__device__ __forceinline__ void track_tile(const TrackParams& p, const int term, const int bx,
                                           const int by, const int bid) {
  Ctrl* __restrict__ ctrl = p.ctrl;
  if (ctrl->status != 0) return;
  const int lane = threadIdx.x;
  const int warp = threadIdx.y;
  constexpr int kR = SPLIT ? kTrackThreadsY : kTrackRows;   // rows between a thread's rows
  const bool icp = SPLIT ? term == 0 : warp < kTrackRows;    // warp-uniform
  const int wrow = SPLIT ? warp : (warp & (kTrackRows - 1));
  const int rs = ctrl->ref_index;
  const int cs = 1 - rs;
  const LevelGeom g = p.g;
  const float* __restrict__ D1 = p.m.depth[cs];
  const float* __restrict__ I1 = p.m.inten[cs];
  const void* __restrict__ A1 = p.m.packA[cs];
  const float* __restrict__ D0 = p.m.depth[rs];
  const void* __restrict__ A0 = p.m.packA[rs];
  const void* __restrict__ B0 = p.m.packB[rs];

  float A[9], t[3];
  const float* xf = icp ? ctrl->xf_icp : ctrl->xf_rgb;
#pragma unroll
  for (int k = 0; k < 9; ++k) A[k] = xf[k];
#pragma unroll
  for (int k = 0; k < 3; ++k) t[k] = xf[9 + k];

  float acc[kSums];
#pragma unroll
  for (int k = 0; k < kSums; ++k) acc[k] = 0.f;

  const int u = bx * kTrackThreadsX + lane;
  const bool col_ok = u < g.w;
  const float dmin = p.depth_min, dmax = p.depth_max;
  // live samples of the thread's row r (zero depth outside the image)
  auto load_live = [&](int r) {
    Live L = {0.f, 0.f, 0.f, 0.f};
    const int v = (by * p.ppt + r) * kR + wrow;
    if (col_ok && v < g.h) {
      const int o = v * g.w + u;
      if (icp) {
        const float4 a = Packs<T>::load_a(A1, D1, o);
        L.d = a.w;
        L.a = a.x;
        L.b = a.y;
        L.c = a.z;
      } else {
        L.d = Packs<T>::depth(A1, D1, o);
        L.a = __ldg(I1 + o);
      }
    }
    return L;
  };
  __shared__ uint8_t s_flag[kTrackRows][kTrackThreadsX];
  Live cur = load_live(0);
  for (int r = 0; r < p.ppt; ++r) {
    const Live nxt = r + 1 < p.ppt ? load_live(r + 1) : Live{0.f, 0.f, 0.f, 0.f};
    const int v = (by * p.ppt + r) * kR + wrow;
    if (kPrefetchRows > 0 && r + kPrefetchRows < p.ppt) {
      const int vf = v + kPrefetchRows * kR;
      if (col_ok && vf < g.h) {
        const int of = vf * g.w + u;
        if (icp) {
          prefetch_l2(static_cast<const char*>(A1) + (size_t)of * Packs<T>::kBytesA);
          prefetch_l2(static_cast<const char*>(A0) + (size_t)of * Packs<T>::kBytesA);
        } else {
          prefetch_l2(I1 + of);
          prefetch_l2(static_cast<const char*>(B0) + (size_t)of * Packs<T>::kBytesB);
        }
      }
    }
    bool ok = false;
    unsigned assoc = 0u;
    if (col_ok && v < g.h && cur.d >= dmin && cur.d <= dmax) {
      ok = icp ? icp_pixel<T, (OPT & kOptDepthWeight) != 0>(p, g, A, t, A0, D0, u, v, cur, acc, &assoc)
               : rgb_pixel<T, (OPT & kOptOcc) != 0>(g, A, t, B0, D0, p.occ_thr, u, v, cur, acc);
    }
    // flag byte: bit 0 ICP, bit 1 photometric, bits 2-5 the ICP association
    const unsigned fbits = ok ? (icp ? 1u | (assoc << 2) : 2u) : 0u;
    if (FLAGS && SPLIT) {    // or-ed into the zeroed flag bytes
      if (ok) {
        const int o = v * g.w + u;
        atomicOr(reinterpret_cast<unsigned int*>(p.flags + (o & ~3)), fbits << (8 * (o & 3)));
      }
    } else if (FLAGS) {      // the two terms' bits combined through shared memory
      if (icp) s_flag[wrow][lane] = (uint8_t)fbits;
      __syncthreads();
      if (!icp && col_ok && v < g.h) p.flags[v * g.w + u] = (uint8_t)(s_flag[wrow][lane] | fbits);
      __syncthreads();
    }
    cur = nxt;
  }

  // ---------------- reduction ----------------
  // Warp: transpose-reduce.  Padded to 32 values, five halving exchanges leave
  // lane l holding the warp sum of value l (31 shuffles instead of 5 per value).
  float w[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) w[k] = k < kSums ? acc[k] : 0.f;
#pragma unroll
  for (int half = 16, off = 16; off > 0; half >>= 1, off >>= 1) {
    const bool hi = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const float send = hi ? w[i] : w[i + half];
      const float keep = hi ? w[i + half] : w[i];
      w[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  __shared__ float s_warp[kTrackThreadsY][32];
  __shared__ bool s_last;
  const int tid = warp * kTrackThreadsX + lane;
  s_warp[warp][lane] = w[0];
  __syncthreads();
  // Block: FP32 sum of each term's warps (four, or eight in a single-term block,
  // whose other term is zero), one FP64 (or FP32) partial per block.  Blocks
  // fold in two deterministic levels: the last block of each group of
  // kFoldGroup blocks sums the group's partials in block order, the last group
  // sums the groups.
  const int grp = bid / kFoldGroup;
  const int ngroups = (p.nblocks + kFoldGroup - 1) / kFoldGroup;
  const int gsize = min(kFoldGroup, p.nblocks - grp * kFoldGroup);
  P* partials = reinterpret_cast<P*>(p.partials);
  P* gpartials = reinterpret_cast<P*>(p.gpartials);
  if (tid < kSumsAll) {
    const int tt = tid / kSums, k = tid - tt * kSums;
    float s = 0.f;                   // zero for the term a single-term block skips
    if (SPLIT) {
      if (tt == term) {
#pragma unroll
        for (int q = 0; q < kTrackThreadsY; ++q) s += s_warp[q][k];
      }
    } else {
#pragma unroll
      for (int q = 0; q < kTrackRows; ++q) s += s_warp[tt * kTrackRows + q][k];
    }
    partials[(int64_t)bid * kSumsAll + tid] = (P)s;
    __threadfence();
  }
  __syncthreads();
  if (tid == 0) s_last = atomicAdd(&p.counters[1 + grp], 1u) == (unsigned)(gsize - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (tid < kSumsAll) {
    P s = 0;
    for (int b = grp * kFoldGroup; b < grp * kFoldGroup + gsize; ++b)
      s += __ldcg(partials + (int64_t)b * kSumsAll + tid);
    gpartials[(int64_t)grp * kSumsAll + tid] = s;
    __threadfence();
  }
  __syncthreads();
  if (tid == 0) {
    p.counters[1 + grp] = 0u;
    s_last = atomicAdd(&p.counters[0], 1u) == (unsigned)(ngroups - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (tid < kSumsAll) {
    P s = 0;
    for (int q = 0; q < ngroups; ++q) s += __ldcg(gpartials + (int64_t)q * kSumsAll + tid);
    ctrl->sums[tid] = (double)s;
  }
  if (tid == 0) p.counters[0] = 0u;
}

template <typename T, typename P, bool FLAGS, int OPT>
__global__ void __launch_bounds__(kTrackThreadsX * kTrackThreadsY)
k_track(TrackParams p) {
  track_tile<T, P, FLAGS, false, OPT>(p, 0, blockIdx.x, blockIdx.y, blockIdx.y * gridDim.x + blockIdx.x);
}

// Tiles of every tracking slot at one level: block -> (slot, tile, term)
// through the block prefix, tile -> (column, row band) in the slot's image.
// Three blocks per SM (80 registers) measured faster than four (64 registers,
// more spill reloads) and than two columns per thread.
// FLAGS (parity entry only): the same kernel that also or-s each pixel's
// validity bits into a.flags (the slot's level image, zeroed before the launch).
template <typename T, typename P, int OPT, bool FLAGS>
__global__ void __launch_bounds__(kTrackThreadsX * kTrackThreadsY, 3)
k_track_batch(const BatchArgs a) {
  const int i = batch_slot(a, blockIdx.x);
  const int slot = a.slot0 + i;
  if (batch_dyn(a, slot).mode != kSlotTrack) return;
  // the slot's parameters, staged once per block in shared memory
  __shared__ TrackParams p;
  const int tid = threadIdx.y * kTrackThreadsX + threadIdx.x;
  if (tid < (int)(sizeof(TrackParams) / 4))
    reinterpret_cast<uint32_t*>(&p)[tid] =
        __ldg(reinterpret_cast<const uint32_t*>(&a.slots[slot].tp[a.level]) + tid);
  __syncthreads();
  if (FLAGS && tid == 0) p.flags = a.flags;
  if (FLAGS) __syncthreads();
  grid_dep_wait();               // the transforms of the preceding Gauss-Newton step
  grid_dep_launch();             // the next step's state-only work may start now
  const int t = blockIdx.x - __ldg(a.start + i);
  const int gx = (p.g.w + kTrackThreadsX - 1) / kTrackThreadsX;
  const int tile = t >> 1;                    // the two terms of a tile are neighbours
  track_tile<T, P, FLAGS, true, OPT>(p, t & 1, tile % gx, tile / gx, t);
}

}  // namespace

// Rows per thread: enough blocks for two per SM on 152 SMs, no more (each block
// pays a reduction and a partial).
int track_default_ppt(int w, int h) {
  const int b1 = track_grid_blocks(w, h, 1);
  int ppt = b1 / 304;
  return ppt < 1 ? 1 : (ppt > 16 ? 16 : ppt);
}

int track_grid_blocks(int w, int h, int ppt) {
  const int gx = (w + kTrackThreadsX - 1) / kTrackThreadsX;
  const int rows = kTrackThreadsY * ppt;
  const int gy = (h + rows - 1) / rows;
  return 2 * gx * gy;
}

int track_mixed_blocks(int w, int h, int ppt) {
  const int gx = (w + kTrackThreadsX - 1) / kTrackThreadsX;
  const int rows = kTrackRows * ppt;
  const int gy = (h + rows - 1) / rows;
  return gx * gy;
}

cudaError_t launch_track(const TrackParams& p0, bool fp16, bool fp32_partials, cudaStream_t s) {
  TrackParams p = p0;
  p.nblocks = track_mixed_blocks(p.g.w, p.g.h, p.ppt);
  const dim3 block(kTrackThreadsX, kTrackThreadsY);
  const int rows = kTrackRows * p.ppt;
  const dim3 grid((p.g.w + kTrackThreadsX - 1) / kTrackThreadsX, (p.g.h + rows - 1) / rows);
  const bool flags = p.flags != nullptr;
  const int opt = (p.occ_thr > 0.f ? kOptOcc : 0) | (p.icp_dw ? kOptDepthWeight : 0);
#define DRI_TRACK_OPT(T, P, O)                                              \
  do {                                                                      \
    if (flags) k_track<T, P, true, O><<<grid, block, 0, s>>>(p);            \
    else k_track<T, P, false, O><<<grid, block, 0, s>>>(p);                 \
  } while (0)
#define DRI_TRACK_LAUNCH(T, P)                                              \
  do {                                                                      \
    if (opt == 0) DRI_TRACK_OPT(T, P, 0);                                   \
    else if (opt == 1) DRI_TRACK_OPT(T, P, 1);                              \
    else if (opt == 2) DRI_TRACK_OPT(T, P, 2);                              \
    else DRI_TRACK_OPT(T, P, 3);                                            \
  } while (0)
  if (fp16) {
    if (fp32_partials) DRI_TRACK_LAUNCH(__half, float);
    else DRI_TRACK_LAUNCH(__half, double);
  } else {
    if (fp32_partials) DRI_TRACK_LAUNCH(float, float);
    else DRI_TRACK_LAUNCH(float, double);
  }
#undef DRI_TRACK_LAUNCH
#undef DRI_TRACK_OPT
  return cudaGetLastError();
}

cudaError_t launch_track_batch(const BatchArgs& a, int blocks, bool fp16, bool fp32_partials,
                               int opt, int priority, bool early, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(kTrackThreadsX, kTrackThreadsY);
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = early ? 1 : 0;
  attr[1].id = cudaLaunchAttributePriority;
  attr[1].val.priority = priority;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
#define DRI_TRACK_BATCH_F(T, P, F)                                                       \
  do {                                                                                   \
    if (opt == 0) return cudaLaunchKernelEx(&cfg, k_track_batch<T, P, 0, F>, a);         \
    if (opt == 1) return cudaLaunchKernelEx(&cfg, k_track_batch<T, P, 1, F>, a);         \
    if (opt == 2) return cudaLaunchKernelEx(&cfg, k_track_batch<T, P, 2, F>, a);         \
    return cudaLaunchKernelEx(&cfg, k_track_batch<T, P, 3, F>, a);                       \
  } while (0)
#define DRI_TRACK_BATCH(T, P)                                                            \
  do {                                                                                   \
    if (a.flags) DRI_TRACK_BATCH_F(T, P, true);                                          \
    DRI_TRACK_BATCH_F(T, P, false);                                                      \
  } while (0)
  if (fp16) {
    if (fp32_partials) DRI_TRACK_BATCH(__half, float);
    DRI_TRACK_BATCH(__half, double);
  }
  if (fp32_partials) DRI_TRACK_BATCH(float, float);
  DRI_TRACK_BATCH(float, double);
#undef DRI_TRACK_BATCH
#undef DRI_TRACK_BATCH_F
}

}  // namespace dri
