// Map building of the tracking pyramid (Sec. IV-D coarse-to-fine scheme; the
// inputs of Eq. 3 and Eq. 4).
//
//   copy_input   level-0 depth / intensity of the live map set from the upload buffer
//   pyr_down     level l from level l-1: depth = mean of the 2x2 samples > 0 (0 if
//                none), intensity = 2x2 mean
//   normals      n = normalise((v(x+1,y) - v) x (v(x,y+1) - v)), facing the camera,
//                invalid (stored as 0) on the last row / column or next to an invalid
//                depth; v = d K^-1 [u, v, 1]^T
//   gradient     central-difference intensity gradient, zero on the one-pixel border
//
// All maps are planar (one plane per component) so a warp reads 128 contiguous
// bytes per plane; normals and gradients are FP32 or, with DRI_FP16_MAPS, FP16.
#include <cuda_fp16.h>

#include "dri_internal.h"

namespace dri {

namespace {

template <typename T>
__device__ __forceinline__ void store_map(T* p, int64_t i, float v);
template <>
__device__ __forceinline__ void store_map<float>(float* p, int64_t i, float v) { p[i] = v; }
template <>
__device__ __forceinline__ void store_map<__half>(__half* p, int64_t i, float v) {
  p[i] = __float2half_rn(v);
}

__global__ void k_copy_input(const float* __restrict__ in_d, const float* __restrict__ in_i,
                             LevelMaps m, const Ctrl* __restrict__ ctrl, int w, int h) {
  const int cs = 1 - ctrl->ref_index;
  const int64_t n = (int64_t)w * h;
  const int64_t n4 = n / 4;
  const float4* d4 = reinterpret_cast<const float4*>(in_d);
  const float4* i4 = reinterpret_cast<const float4*>(in_i);
  float4* od = reinterpret_cast<float4*>(m.depth[cs]);
  float4* oi = reinterpret_cast<float4*>(m.inten[cs]);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n4;
       k += (int64_t)gridDim.x * blockDim.x) {
    od[k] = __ldg(d4 + k);
    oi[k] = __ldg(i4 + k);
  }
  for (int64_t k = n4 * 4 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    m.depth[cs][k] = in_d[k];
    m.inten[cs][k] = in_i[k];
  }
}

__global__ void k_pyr_down(LevelMaps fine, LevelMaps coarse, const Ctrl* __restrict__ ctrl,
                           int wf, int hf, int wc, int hc) {
  const int cs = 1 - ctrl->ref_index;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= wc || y >= hc) return;
  const float* D = fine.depth[cs];
  const float* I = fine.inten[cs];
  const int64_t i0 = (int64_t)(2 * y) * wf + 2 * x;
  const int64_t i1 = i0 + wf;
  const float2 da = __ldg(reinterpret_cast<const float2*>(D + i0));
  const float2 db = __ldg(reinterpret_cast<const float2*>(D + i1));
  const float2 ia = __ldg(reinterpret_cast<const float2*>(I + i0));
  const float2 ib = __ldg(reinterpret_cast<const float2*>(I + i1));
  float s = 0.f;
  int n = 0;
  if (da.x > 0.f) { s += da.x; ++n; }
  if (da.y > 0.f) { s += da.y; ++n; }
  if (db.x > 0.f) { s += db.x; ++n; }
  if (db.y > 0.f) { s += db.y; ++n; }
  const int64_t o = (int64_t)y * wc + x;
  coarse.depth[cs][o] = n ? s / (float)n : 0.f;
  coarse.inten[cs][o] = ((ia.x + ia.y) + (ib.x + ib.y)) * 0.25f;
}

template <typename T>
__global__ void k_normals(LevelMaps m, const Ctrl* __restrict__ ctrl, LevelGeom g, float dmin,
                          float dmax, int which) {
  const int set = which < 0 ? 1 - ctrl->ref_index : which;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= g.w || y >= g.h) return;
  const float* D = m.depth[set];
  T* N = reinterpret_cast<T*>(m.normal[set]);
  const int64_t o = (int64_t)y * g.w + x;
  float nx = 0.f, ny = 0.f, nz = 0.f;
  if (x + 1 < g.w && y + 1 < g.h) {
    const float d0 = __ldg(D + o);
    const float d1 = __ldg(D + o + 1);
    const float d2 = __ldg(D + o + g.w);
    const bool ok = d0 >= dmin && d0 <= dmax && d1 >= dmin && d1 <= dmax && d2 >= dmin && d2 <= dmax;
    if (ok) {
      const float rx = ((float)x - g.cx) * g.ifx;
      const float ry = ((float)y - g.cy) * g.ify;
      const float rx1 = ((float)(x + 1) - g.cx) * g.ifx;
      const float ry2 = ((float)(y + 1) - g.cy) * g.ify;
      // forward differences of v = d * ray, written so no large terms cancel
      const float e1 = d1 - d0, e2 = d2 - d0;
      const float ax = fmaf(e1, rx1, d0 * g.ifx), ay = e1 * ry, az = e1;
      const float bx = e2 * rx, by = fmaf(e2, ry2, d0 * g.ify), bz = e2;
      float cx = ay * bz - az * by;
      float cy = az * bx - ax * bz;
      float cz = ax * by - ay * bx;
      const float n2 = cx * cx + cy * cy + cz * cz;
      if (n2 > 0.f) {
        const float inv = rsqrtf(n2);
        cx *= inv;
        cy *= inv;
        cz *= inv;
        if (cx * rx + cy * ry + cz > 0.f) {   // sign of n . v (v = d0 * ray, d0 > 0)
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
  store_map<T>(N, o, nx);
  store_map<T>(N, o + m.plane, ny);
  store_map<T>(N, o + 2 * m.plane, nz);
}

template <typename T>
__global__ void k_gradient(LevelMaps m, const Ctrl* __restrict__ ctrl, int w, int h) {
  // the set that is (or just became) the reference
  const int set = ctrl->ref_index;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= w || y >= h) return;
  const float* I = m.inten[set];
  T* G = reinterpret_cast<T*>(m.grad[set]);
  const int64_t o = (int64_t)y * w + x;
  float gx = 0.f, gy = 0.f;
  if (x > 0 && y > 0 && x + 1 < w && y + 1 < h) {
    gx = 0.5f * (__ldg(I + o + 1) - __ldg(I + o - 1));
    gy = 0.5f * (__ldg(I + o + w) - __ldg(I + o - w));
  }
  store_map<T>(G, o, gx);
  store_map<T>(G, o + m.plane, gy);
}

inline dim3 grid2(int w, int h, dim3 b) { return dim3((w + b.x - 1) / b.x, (h + b.y - 1) / b.y); }

}  // namespace

cudaError_t launch_copy_input(const float* in_d, const float* in_i, const LevelMaps& m0,
                              const Ctrl* ctrl, int w, int h, cudaStream_t s) {
  const int64_t n4 = ((int64_t)w * h + 3) / 4;
  int blocks = (int)((n4 + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_copy_input<<<blocks, 256, 0, s>>>(in_d, in_i, m0, ctrl, w, h);
  return cudaGetLastError();
}

cudaError_t launch_pyr_down(const LevelMaps& fine, const LevelMaps& coarse, const Ctrl* ctrl,
                            int wf, int hf, int wc, int hc, cudaStream_t s) {
  const dim3 b(32, 8);
  k_pyr_down<<<grid2(wc, hc, b), b, 0, s>>>(fine, coarse, ctrl, wf, hf, wc, hc);
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
