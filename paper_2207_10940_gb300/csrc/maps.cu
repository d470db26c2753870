// Map building of the tracking pyramid (Sec. IV-D coarse-to-fine scheme; the
// inputs of Eq. 3 and Eq. 4).
//
//   copy         level-0 depth / intensity of the live map set from the frame's images
//   pyr_down     level l from level l-1: depth = mean of the 2x2 samples > 0 (0 if
//                none), intensity = 2x2 mean
//   normals      n = normalise((v(x+1,y) - v) x (v(x,y+1) - v)), facing the camera,
//                invalid (stored as 0) on the last row / column or next to an invalid
//                depth; v = d K^-1 [u, v, 1]^T; written with the depth as pack A
//   gradient     central-difference intensity gradient, zero on the one-pixel border;
//                written with the intensity as pack B
//
// Depth and intensity are FP32 planes; the packs (packs.cuh) hold FP32 or, with
// DRI_FP16_MAPS, FP16 normals and gradients.
// The batched kernels cover the images of every slot of a plan in one launch;
// the single-image normal and gradient kernels serve the allocation-free entry.
#include <cuda_fp16.h>

#include "dri_internal.h"
#include "packs.cuh"

namespace dri {

namespace {

// Level-0 copy of one 128 x 8 tile: each thread moves 4 pixels of a row, as one
// 16-byte load and store when both rows allow it.
__global__ void __launch_bounds__(256) k_copy_batch(const BatchArgs a) {
  const int i = batch_slot(a, blockIdx.x);
  const int slot = a.slot0 + i;
  const SlotDyn& d = batch_dyn(a, slot);
  if (d.mode == kSlotIdle) return;
  const TrackParams& tp = a.slots[slot].tp[0];
  const int w = tp.g.w, h = tp.g.h;
  const int cs = 1 - tp.ctrl->ref_index;
  const int t = blockIdx.x - __ldg(a.start + i);
  const int gx = (w + kCopyTileW - 1) / kCopyTileW;
  const int x = (t % gx) * kCopyTileW + threadIdx.x * 4;
  const int y = (t / gx) * kCopyTileH + threadIdx.y;
  if (x >= w || y >= h) return;
  const float* sd = d.src_depth + (int64_t)y * d.pitch + x;
  const float* si = d.src_inten + (int64_t)y * d.pitch + x;
  float* od = tp.m.depth[cs] + (int64_t)y * w + x;
  float* oi = tp.m.inten[cs] + (int64_t)y * w + x;
  const uintptr_t al = (uintptr_t)sd | (uintptr_t)si | (uintptr_t)od | (uintptr_t)oi;
  if (x + 4 <= w && (al & 15) == 0) {
    *reinterpret_cast<float4*>(od) = __ldg(reinterpret_cast<const float4*>(sd));
    *reinterpret_cast<float4*>(oi) = __ldg(reinterpret_cast<const float4*>(si));
  } else {
    const int n = min(4, w - x);
    for (int k = 0; k < n; ++k) {
      od[k] = __ldg(sd + k);
      oi[k] = __ldg(si + k);
    }
  }
}

__device__ __forceinline__ void pyr_down_px(const LevelMaps& fine, const LevelMaps& coarse, int cs,
                                            int wf, int wc, int x, int y) {
  const float* D = fine.depth[cs];
  const float* I = fine.inten[cs];
  const int64_t i0 = (int64_t)(2 * y) * wf + 2 * x;
  const int64_t i1 = i0 + wf;
  float da0, da1, db0, db1, ia0, ia1, ib0, ib1;
  if ((wf & 1) == 0) {                 // rows of even width keep the 2x2 pairs 8-byte aligned
    const float2 da = __ldg(reinterpret_cast<const float2*>(D + i0));
    const float2 db = __ldg(reinterpret_cast<const float2*>(D + i1));
    const float2 ia = __ldg(reinterpret_cast<const float2*>(I + i0));
    const float2 ib = __ldg(reinterpret_cast<const float2*>(I + i1));
    da0 = da.x; da1 = da.y; db0 = db.x; db1 = db.y;
    ia0 = ia.x; ia1 = ia.y; ib0 = ib.x; ib1 = ib.y;
  } else {
    da0 = __ldg(D + i0); da1 = __ldg(D + i0 + 1); db0 = __ldg(D + i1); db1 = __ldg(D + i1 + 1);
    ia0 = __ldg(I + i0); ia1 = __ldg(I + i0 + 1); ib0 = __ldg(I + i1); ib1 = __ldg(I + i1 + 1);
  }
  float s = 0.f;
  int n = 0;
  if (da0 > 0.f) { s += da0; ++n; }
  if (da1 > 0.f) { s += da1; ++n; }
  if (db0 > 0.f) { s += db0; ++n; }
  if (db1 > 0.f) { s += db1; ++n; }
  const int64_t o = (int64_t)y * wc + x;
  coarse.depth[cs][o] = n ? s / (float)n : 0.f;
  coarse.inten[cs][o] = ((ia0 + ia1) + (ib0 + ib1)) * 0.25f;
}

template <typename T>
__device__ __forceinline__ void normal_px(const LevelMaps& m, int set, const LevelGeom& g,
                                          float dmin, float dmax, int x, int y) {
  const float* D = m.depth[set];
  const int o = y * g.w + x;
  const float d0 = __ldg(D + o);
  float nx = 0.f, ny = 0.f, nz = 0.f;
  if (x + 1 < g.w && y + 1 < g.h) {
    const float d1 = __ldg(D + o + 1);
    const float d2 = __ldg(D + o + g.w);
    const bool ok = d0 >= dmin && d0 <= dmax && d1 >= dmin && d1 <= dmax && d2 >= dmin && d2 <= dmax;
    if (ok) {
      const float rx = ((float)x - g.cx) * g.ifx;
      const float ry = ((float)y - g.cy) * g.ify;
      const float rx1 = ((float)(x + 1) - g.cx) * g.ifx;
      const float ry2 = ((float)(y + 1) - g.cy) * g.ify;
      // forward differences of v = d * ray, written so no large terms cancel; every
      // product and sum is spelled out (fmaf / __fmul_rn) so that no kernel this is
      // inlined into contracts it differently: all map kernels give identical bits
      const float e1 = d1 - d0, e2 = d2 - d0;
      const float ax = fmaf(e1, rx1, __fmul_rn(d0, g.ifx)), ay = __fmul_rn(e1, ry), az = e1;
      const float bx = __fmul_rn(e2, rx), by = fmaf(e2, ry2, __fmul_rn(d0, g.ify)), bz = e2;
      float cx = fmaf(ay, bz, -__fmul_rn(az, by));
      float cy = fmaf(az, bx, -__fmul_rn(ax, bz));
      float cz = fmaf(ax, by, -__fmul_rn(ay, bx));
      const float n2 = fmaf(cx, cx, fmaf(cy, cy, __fmul_rn(cz, cz)));
      if (n2 > 0.f) {
        const float inv = rsqrtf(n2);
        cx = __fmul_rn(cx, inv);
        cy = __fmul_rn(cy, inv);
        cz = __fmul_rn(cz, inv);
        if (fmaf(cx, rx, fmaf(cy, ry, cz)) > 0.f) {   // sign of n . v (v = d0 * ray, d0 > 0)
          cx = -cx;
          cy = -cy;
          cz = -cz;
        }
        nx = cx;
        ny = cy;
        nz = cz;
      }
    }
  }
  Packs<T>::store_a(m.packA[set], o, nx, ny, nz, d0);
}

template <typename T>
__device__ __forceinline__ void gradient_px(const LevelMaps& m, int set, int w, int h, int x, int y) {
  const float* I = m.inten[set];
  const int o = y * w + x;
  float gx = 0.f, gy = 0.f;
  if (x > 0 && y > 0 && x + 1 < w && y + 1 < h) {
    gx = 0.5f * (__ldg(I + o + 1) - __ldg(I + o - 1));
    gy = 0.5f * (__ldg(I + o + w) - __ldg(I + o - w));
  }
  Packs<T>::store_b(m.packB[set], o, __ldg(I + o), gx, gy, __ldg(m.depth[set] + o));
}

// Block -> (slot, 32 x 8 kMapRows tile of the slot's level-`a.level` image):
// the thread's column x and first row y (its rows are y, y + 8, ...); false for
// an idle slot.  w, h: the level's size.
__device__ __forceinline__ bool map_tile(const BatchArgs& a, int* slot, int* x, int* y, int* w,
                                         int* h) {
  const int i = batch_slot(a, blockIdx.x);
  *slot = a.slot0 + i;
  if (batch_dyn(a, *slot).mode == kSlotIdle) return false;
  const LevelGeom& g = a.slots[*slot].tp[a.level].g;
  const int t = blockIdx.x - __ldg(a.start + i);
  const int gx = (g.w + kMapTileW - 1) / kMapTileW;
  *x = (t % gx) * kMapTileW + threadIdx.x;
  *y = (t / gx) * kMapTileH * kMapRows + threadIdx.y;
  *w = g.w;
  *h = g.h;
  return true;
}

__global__ void __launch_bounds__(256) k_pyr_down_batch(const BatchArgs a) {
  int slot, x, y, w, h;
  if (!map_tile(a, &slot, &x, &y, &w, &h) || x >= w) return;
  const SlotStatic& st = a.slots[slot];
  const int cs = 1 - st.tp[0].ctrl->ref_index;
#pragma unroll
  for (int k = 0; k < kMapRows; ++k, y += kMapTileH)
    if (y < h) pyr_down_px(st.tp[a.level - 1].m, st.tp[a.level].m, cs, st.tp[a.level - 1].g.w, w, x, y);
}

template <typename T>
__global__ void __launch_bounds__(256) k_normals_batch(const BatchArgs a) {
  int slot, x, y, w, h;
  if (!map_tile(a, &slot, &x, &y, &w, &h) || x >= w) return;
  const TrackParams& tp = a.slots[slot].tp[a.level];
  const int cs = 1 - tp.ctrl->ref_index;
#pragma unroll
  for (int k = 0; k < kMapRows; ++k, y += kMapTileH)
    if (y < h) normal_px<T>(tp.m, cs, tp.g, tp.depth_min, tp.depth_max, x, y);
}

template <typename T>
__global__ void __launch_bounds__(256) k_gradient_batch(const BatchArgs a) {
  int slot, x, y, w, h;
  if (!map_tile(a, &slot, &x, &y, &w, &h) || x >= w) return;
  const TrackParams& tp = a.slots[slot].tp[a.level];
  // the frame's own map set, which becomes the reference at the frame end
  // (launched before it)
  const int cs = 1 - tp.ctrl->ref_index;
#pragma unroll
  for (int k = 0; k < kMapRows; ++k, y += kMapTileH)
    if (y < h) gradient_px<T>(tp.m, cs, w, h, x, y);
}

template <typename T>
__global__ void k_normals(LevelMaps m, const Ctrl* __restrict__ ctrl, LevelGeom g, float dmin,
                          float dmax, int which) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= g.w || y >= g.h) return;
  normal_px<T>(m, which < 0 ? 1 - ctrl->ref_index : which, g, dmin, dmax, x, y);
}

template <typename T>
__global__ void k_gradient(LevelMaps m, const Ctrl* __restrict__ ctrl, int w, int h) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= w || y >= h) return;
  gradient_px<T>(m, ctrl->ref_index, w, h, x, y);
}


// ---- uploaded reference (a model prediction rendered at T_ref) ----
// Level 0: per pixel, the vertex and normal moved into the reference camera in
// FP64 (v = R^T (V - r), n = R^T N); a zero normal means no surface (depth 0);
// the normal is kept where the depth is in [dmin, dmax].
template <typename T>
__global__ void k_ref_level0(LevelMaps m, const Ctrl* __restrict__ ctrl, LevelGeom g, float dmin,
                             float dmax, RefUpload up) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= g.w || y >= g.h) return;
  const int set = ctrl->ref_index;
  const int64_t src = (int64_t)y * up.pitch + x;
  const float* V = up.V + 3 * src;
  const float* N = up.N + 3 * src;
  const double vx = (double)__ldg(V) - up.r[0], vy = (double)__ldg(V + 1) - up.r[1],
               vz = (double)__ldg(V + 2) - up.r[2];
  const double nx = __ldg(N), ny = __ldg(N + 1), nz = __ldg(N + 2);
  const bool surf = nx != 0.0 || ny != 0.0 || nz != 0.0;
  const double* R = up.R;
  const float d = surf ? (float)(R[2] * vx + R[5] * vy + R[8] * vz) : 0.f;
  const bool keep = surf && d >= dmin && d <= dmax;
  const float cx = keep ? (float)(R[0] * nx + R[3] * ny + R[6] * nz) : 0.f;
  const float cy = keep ? (float)(R[1] * nx + R[4] * ny + R[7] * nz) : 0.f;
  const float cz = keep ? (float)(R[2] * nx + R[5] * ny + R[8] * nz) : 0.f;
  const int o = y * g.w + x;
  m.depth[set][o] = d;
  m.inten[set][o] = __ldg(up.I + src);
  Packs<T>::store_a(m.packA[set], o, cx, cy, cz, d);
}

// Level l from l - 1 of the reference set: depth (mean of the samples > 0) and
// intensity as for a live frame, the normal as the mean of the non-zero normals
// of the 2x2 block, renormalised, kept where the level's depth is in range.
template <typename T>
__global__ void k_ref_down(LevelMaps fine, LevelMaps coarse, const Ctrl* __restrict__ ctrl, int wf,
                           int wc, int hc, float dmin, float dmax) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= wc || y >= hc) return;
  const int set = ctrl->ref_index;
  pyr_down_px(fine, coarse, set, wf, wc, x, y);
  const int o = y * wc + x;
  const float d = coarse.depth[set][o];
  float sx = 0.f, sy = 0.f, sz = 0.f;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int f = (2 * y + (k >> 1)) * wf + 2 * x + (k & 1);
    const float4 n = Packs<T>::load_a(fine.packA[set], fine.depth[set], f);
    sx += n.x;                                   // zero normals add nothing
    sy += n.y;
    sz += n.z;
  }
  const float n2 = fmaf(sx, sx, fmaf(sy, sy, __fmul_rn(sz, sz)));
  float nx = 0.f, ny = 0.f, nz = 0.f;
  if (n2 > 0.f && d >= dmin && d <= dmax) {
    const float inv = rsqrtf(n2);
    nx = __fmul_rn(sx, inv);
    ny = __fmul_rn(sy, inv);
    nz = __fmul_rn(sz, inv);
  }
  Packs<T>::store_a(coarse.packA[set], o, nx, ny, nz, d);
}

__global__ void k_ref_pose(Ctrl* __restrict__ ctrl, RefUpload up) {
  const int i = threadIdx.x;
  if (i < 9) ctrl->Rref[i] = up.R[i];
  if (i < 3) ctrl->rref[i] = up.r[i];
}

inline dim3 grid2(int w, int h, dim3 b) { return dim3((w + b.x - 1) / b.x, (h + b.y - 1) / b.y); }

}  // namespace

cudaError_t launch_copy_batch(const BatchArgs& a, int blocks, cudaStream_t s) {
  k_copy_batch<<<blocks, dim3(kCopyTileW / 4, kCopyTileH), 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_pyr_down_batch(const BatchArgs& a, int blocks, cudaStream_t s) {
  k_pyr_down_batch<<<blocks, dim3(kMapTileW, kMapTileH), 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_normals_batch(const BatchArgs& a, int blocks, bool fp16, cudaStream_t s) {
  if (fp16) k_normals_batch<__half><<<blocks, dim3(kMapTileW, kMapTileH), 0, s>>>(a);
  else k_normals_batch<float><<<blocks, dim3(kMapTileW, kMapTileH), 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_gradient_batch(const BatchArgs& a, int blocks, bool fp16, cudaStream_t s) {
  if (fp16) k_gradient_batch<__half><<<blocks, dim3(kMapTileW, kMapTileH), 0, s>>>(a);
  else k_gradient_batch<float><<<blocks, dim3(kMapTileW, kMapTileH), 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_normals(const LevelMaps& m, const Ctrl* ctrl, const LevelGeom& g, float dmin,
                           float dmax, bool fp16, int which_set, cudaStream_t s) {
  const dim3 b(32, 8);
  if (fp16)
    k_normals<__half><<<grid2(g.w, g.h, b), b, 0, s>>>(m, ctrl, g, dmin, dmax, which_set);
  else
    k_normals<float><<<grid2(g.w, g.h, b), b, 0, s>>>(m, ctrl, g, dmin, dmax, which_set);
  return cudaGetLastError();
}

cudaError_t launch_gradient(const LevelMaps& m, const Ctrl* ctrl, int w, int h, bool fp16,
                            cudaStream_t s) {
  const dim3 b(32, 8);
  if (fp16)
    k_gradient<__half><<<grid2(w, h, b), b, 0, s>>>(m, ctrl, w, h);
  else
    k_gradient<float><<<grid2(w, h, b), b, 0, s>>>(m, ctrl, w, h);
  return cudaGetLastError();
}

}  // namespace dri

namespace dri {

cudaError_t launch_upload_reference(const LevelMaps* m, const LevelGeom* g, int levels, Ctrl* ctrl,
                                    float dmin, float dmax, bool fp16, const RefUpload& up,
                                    cudaStream_t s) {
  const dim3 b(32, 8);
  if (fp16) k_ref_level0<__half><<<grid2(g[0].w, g[0].h, b), b, 0, s>>>(m[0], ctrl, g[0], dmin, dmax, up);
  else k_ref_level0<float><<<grid2(g[0].w, g[0].h, b), b, 0, s>>>(m[0], ctrl, g[0], dmin, dmax, up);
  for (int l = 1; l < levels; ++l) {
    const dim3 gr = grid2(g[l].w, g[l].h, b);
    if (fp16) k_ref_down<__half><<<gr, b, 0, s>>>(m[l - 1], m[l], ctrl, g[l - 1].w, g[l].w, g[l].h, dmin, dmax);
    else k_ref_down<float><<<gr, b, 0, s>>>(m[l - 1], m[l], ctrl, g[l - 1].w, g[l].w, g[l].h, dmin, dmax);
  }
  for (int l = 0; l < levels; ++l) {
    if (fp16) k_gradient<__half><<<grid2(g[l].w, g[l].h, b), b, 0, s>>>(m[l], ctrl, g[l].w, g[l].h);
    else k_gradient<float><<<grid2(g[l].w, g[l].h, b), b, 0, s>>>(m[l], ctrl, g[l].w, g[l].h);
  }
  k_ref_pose<<<1, 32, 0, s>>>(ctrl, up);
  return cudaGetLastError();
}

}  // namespace dri
