// Fused per-pixel Gauss-Newton linearisation of the photometric (Eq. 3) and
// point-to-plane ICP (Eq. 4) terms at one pyramid level, block-reduced into the
// normal equations of Eq. 7 (Sec. IV-B, IV-D).
//
// One thread handles `ppt` pixels of one column of a 32-wide tile (a warp reads
// 128 contiguous bytes per map plane).  Per pixel, in FP32:
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
// back in FP64.  Each term accumulates 29 values per thread (upper J J^T, J e,
// e^2, count) in FP32, reduced by warp shuffles and a shared-memory tree to one
// FP64 (or FP32) partial per block; the partials are folded in two fixed-order
// levels (groups of blocks, then the groups) into ctrl->sums: deterministic, no
// float atomics.
#include <cuda_fp16.h>

#include "dri_internal.h"

namespace dri {

namespace {

template <typename T>
__device__ __forceinline__ float load_map(const T* p, int64_t i);
template <>
__device__ __forceinline__ float load_map<float>(const float* p, int64_t i) { return __ldg(p + i); }
template <>
__device__ __forceinline__ float load_map<__half>(const __half* p, int64_t i) {
  return __half2float(__ldg(p + i));
}

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

template <typename T, typename P, bool FLAGS>
__global__ void __launch_bounds__(kTrackThreadsX * kTrackThreadsY)
k_track(TrackParams p) {
  Ctrl* __restrict__ ctrl = p.ctrl;
  if (ctrl->status != 0) return;
  const int rs = ctrl->ref_index;
  const int cs = 1 - rs;
  const LevelGeom g = p.g;
  const int64_t plane = p.m.plane;
  const float* __restrict__ D1 = p.m.depth[cs];
  const float* __restrict__ I1 = p.m.inten[cs];
  const T* __restrict__ N1 = reinterpret_cast<const T*>(p.m.normal[cs]);
  const float* __restrict__ D0 = p.m.depth[rs];
  const float* __restrict__ I0 = p.m.inten[rs];
  const T* __restrict__ N0 = reinterpret_cast<const T*>(p.m.normal[rs]);
  const T* __restrict__ G0 = reinterpret_cast<const T*>(p.m.grad[rs]);

  float Ai[9], ti[3], Ar[9], tr[3];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    Ai[k] = ctrl->xf_icp[k];
    Ar[k] = ctrl->xf_rgb[k];
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    ti[k] = ctrl->xf_icp[9 + k];
    tr[k] = ctrl->xf_rgb[9 + k];
  }

  float acc[kSumsAll];
#pragma unroll
  for (int k = 0; k < kSumsAll; ++k) acc[k] = 0.f;

  const int u = blockIdx.x * kTrackThreadsX + threadIdx.x;
  for (int r = 0; r < p.ppt; ++r) {
    const int v = (blockIdx.y * p.ppt + r) * kTrackThreadsY + threadIdx.y;
    if (u >= g.w || v >= g.h) continue;
    const int64_t o = (int64_t)v * g.w + u;
    const float d = __ldg(D1 + o);
    uint8_t flag = 0;
    if (d >= p.depth_min && d <= p.depth_max) {
      const float rx = ((float)u - g.cx) * g.ifx;
      const float ry = ((float)v - g.cy) * g.ify;
      const float px = d * rx, py = d * ry, pz = d;

      // ---------------- photometric term (Eq. 3) ----------------
      {
        const float ex = fmaf(Ar[0], px, fmaf(Ar[1], py, fmaf(Ar[2], pz, tr[0])));
        const float ey = fmaf(Ar[3], px, fmaf(Ar[4], py, fmaf(Ar[5], pz, tr[1])));
        const float ez = fmaf(Ar[6], px, fmaf(Ar[7], py, fmaf(Ar[8], pz, tr[2])));
        const float z = d + ez;
        if (z > 0.f) {
          const float iz = 1.f / z;
          // displacement of the projection from (u, v): small, so FP32 keeps it to
          // ~1e-6 px, and integer parts of the position stay exact
          const float sxp = g.fx * (fmaf(-rx, ez, ex) * iz);
          const float syp = g.fy * (fmaf(-ry, ez, ey) * iz);
          const float fxp = floorf(sxp), fyp = floorf(syp);
          const bool sane = fabsf(sxp) < 1e7f && fabsf(syp) < 1e7f;   // int conversion in range
          const int xb = sane ? u + (int)fxp : -1, yb = sane ? v + (int)fyp : -1;
          if (xb >= 0 && xb < g.w - 1 && yb >= 0 && yb < g.h - 1) {
            const float ax = sxp - fxp, ay = syp - fyp;
            const int64_t q = (int64_t)yb * g.w + xb;
            const float w00 = (1.f - ax) * (1.f - ay), w01 = ax * (1.f - ay);
            const float w10 = (1.f - ax) * ay, w11 = ax * ay;
            const float iv = w00 * __ldg(I0 + q) + w01 * __ldg(I0 + q + 1) +
                             w10 * __ldg(I0 + q + g.w) + w11 * __ldg(I0 + q + g.w + 1);
            const float gx = w00 * load_map(G0, q) + w01 * load_map(G0, q + 1) +
                             w10 * load_map(G0, q + g.w) + w11 * load_map(G0, q + g.w + 1);
            const float gy = w00 * load_map(G0, plane + q) + w01 * load_map(G0, plane + q + 1) +
                             w10 * load_map(G0, plane + q + g.w) +
                             w11 * load_map(G0, plane + q + g.w + 1);
            const float e = iv - __ldg(I1 + o);
            const float a0 = g.fx * gx * iz, a1 = g.fy * gy * iz;
            const float a2 = -(gx * (((float)u - g.cx) + sxp) + gy * (((float)v - g.cy) + syp)) * iz;
            const float sx = px + (ex - tr[0]), sy = py + (ey - tr[1]), sz = pz + (ez - tr[2]);
            float J[6] = {a0, a1, a2, sy * a2 - sz * a1, sz * a0 - sx * a2, sx * a1 - sy * a0};
            accumulate(acc + kSums, J, e);
            flag |= 2;
          }
        }
      }

      // ---------------- ICP term (Eq. 4) ----------------
      const float n1x = load_map(N1, o), n1y = load_map(N1, plane + o), n1z = load_map(N1, 2 * plane + o);
      if (n1x != 0.f || n1y != 0.f || n1z != 0.f) {
        const float ex = fmaf(Ai[0], px, fmaf(Ai[1], py, fmaf(Ai[2], pz, ti[0])));
        const float ey = fmaf(Ai[3], px, fmaf(Ai[4], py, fmaf(Ai[5], pz, ti[1])));
        const float ez = fmaf(Ai[6], px, fmaf(Ai[7], py, fmaf(Ai[8], pz, ti[2])));
        const float z = d + ez;
        if (z > 0.f) {
          const float iz = 1.f / z;
          const float sxp = g.fx * (fmaf(-rx, ez, ex) * iz);
          const float syp = g.fy * (fmaf(-ry, ez, ey) * iz);
          const bool sane = fabsf(sxp) < 1e7f && fabsf(syp) < 1e7f;
          const int xi = sane ? u + (int)floorf(sxp + 0.5f) : -1;
          const int yi = sane ? v + (int)floorf(syp + 0.5f) : -1;
          if (xi >= 0 && xi < g.w && yi >= 0 && yi < g.h) {
            const int64_t q = (int64_t)yi * g.w + xi;
            const float Nx = load_map(N0, q), Ny = load_map(N0, plane + q), Nz = load_map(N0, 2 * plane + q);
            if (Nx != 0.f || Ny != 0.f || Nz != 0.f) {
              const float dr = __ldg(D0 + q);
              const float Vx = dr * (((float)xi - g.cx) * g.ifx), Vy = dr * (((float)yi - g.cy) * g.ify);
              const float dx = (px - Vx) + ex, dy = (py - Vy) + ey, dz = (pz - dr) + ez;
              const float dist2 = dx * dx + dy * dy + dz * dz;
              const float mx = n1x + (Ai[0] * n1x + Ai[1] * n1y + Ai[2] * n1z);
              const float my = n1y + (Ai[3] * n1x + Ai[4] * n1y + Ai[5] * n1z);
              const float mz = n1z + (Ai[6] * n1x + Ai[7] * n1y + Ai[8] * n1z);
              const float cosang = mx * Nx + my * Ny + mz * Nz;
              if (dist2 < p.icp_dist2 && cosang > p.icp_cos) {
                const float e = Nx * dx + Ny * dy + Nz * dz;
                const float sx = px + (ex - ti[0]), sy = py + (ey - ti[1]), sz = pz + (ez - ti[2]);
                float J[6] = {Nx, Ny, Nz, sy * Nz - sz * Ny, sz * Nx - sx * Nz, sx * Ny - sy * Nx};
                accumulate(acc, J, e);
                flag |= 1;
              }
            }
          }
        }
      }
    }
    if (FLAGS) p.flags[o] = flag;
  }

  // ---------------- reduction ----------------
  // Warp: transpose-reduce.  Padded to 64 values, five halving exchanges leave
  // lane l holding the warp sums of values 2l and 2l + 1 (62 shuffles instead of
  // 5 per value).
  float v[64];
#pragma unroll
  for (int k = 0; k < 64; ++k) v[k] = k < kSumsAll ? acc[k] : 0.f;
  const int lane = threadIdx.x;
#pragma unroll
  for (int half = 32, off = 16; off > 0; half >>= 1, off >>= 1) {
    const bool hi = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const float send = hi ? v[i] : v[i + half];
      const float keep = hi ? v[i + half] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  __shared__ float s_warp[kTrackThreadsY][64];
  __shared__ bool s_last;
  const int tid = threadIdx.y * kTrackThreadsX + threadIdx.x;
  s_warp[threadIdx.y][2 * lane] = v[0];
  s_warp[threadIdx.y][2 * lane + 1] = v[1];
  __syncthreads();
  // Block: FP32 sum of the warps, one FP64 (or FP32) partial per block.  Blocks fold
  // in two deterministic levels: the last block of each group of kFoldGroup blocks
  // sums the group's partials in block order, the last group sums the groups.
  const int bid = blockIdx.y * gridDim.x + blockIdx.x;
  const int grp = bid / kFoldGroup;
  const int ngroups = (p.nblocks + kFoldGroup - 1) / kFoldGroup;
  const int gsize = min(kFoldGroup, p.nblocks - grp * kFoldGroup);
  P* partials = reinterpret_cast<P*>(p.partials);
  P* gpartials = reinterpret_cast<P*>(p.gpartials);
  if (tid < kSumsAll) {
    float s = 0.f;
#pragma unroll
    for (int w = 0; w < kTrackThreadsY; ++w) s += s_warp[w][tid];
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
    for (int g = 0; g < ngroups; ++g) s += __ldcg(gpartials + (int64_t)g * kSumsAll + tid);
    ctrl->sums[tid] = (double)s;
  }
  if (tid == 0) p.counters[0] = 0u;
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
  return gx * gy;
}

cudaError_t launch_track(const TrackParams& p, bool fp16, bool fp32_partials, cudaStream_t s) {
  const dim3 block(kTrackThreadsX, kTrackThreadsY);
  const int rows = kTrackThreadsY * p.ppt;
  const dim3 grid((p.g.w + kTrackThreadsX - 1) / kTrackThreadsX, (p.g.h + rows - 1) / rows);
  const bool flags = p.flags != nullptr;
#define DRI_TRACK_LAUNCH(T, P)                                              \
  do {                                                                      \
    if (flags) k_track<T, P, true><<<grid, block, 0, s>>>(p);               \
    else k_track<T, P, false><<<grid, block, 0, s>>>(p);                    \
  } while (0)
  if (fp16) {
    if (fp32_partials) DRI_TRACK_LAUNCH(__half, float);
    else DRI_TRACK_LAUNCH(__half, double);
  } else {
    if (fp32_partials) DRI_TRACK_LAUNCH(float, float);
    else DRI_TRACK_LAUNCH(float, double);
  }
#undef DRI_TRACK_LAUNCH
  return cudaGetLastError();
}

}  // namespace dri
