// Per-pixel map packs of the pixel kernel (one vector load per gather).
//
//   pack A  normal and depth, the ICP term's samples (Eq. 4):
//           FP32 maps: float4 {n_x, n_y, n_z, d}
//           FP16 maps: 8 bytes {half n_x, n_y, n_z, 0}; the depth comes from the
//                      FP32 depth plane (half precision would move a point at 8 m
//                      by 4 mm)
//   pack B  intensity and its gradient, the photometric reference (Eq. 3):
//           FP32 maps: float4 {I, g_x, g_y, d} (d: the reference depth, which the
//                      occlusion test reads from the bilinear tap nearest to the
//                      warped point, no extra load)
//           FP16 maps: 8 bytes {float I, half g_x, half g_y} (the occlusion test
//                      reads the depth plane)
//
// An invalid normal is stored as zero.  The live frame needs pack A (and the
// intensity plane); pack B is written when a frame becomes the reference.
#pragma once

#include <cuda_fp16.h>

namespace dri {

template <typename T>
struct Packs;

template <>
struct Packs<float> {
  static constexpr int kBytesA = 16, kBytesB = 16;
  static constexpr bool kDepthInB = true;
  __device__ __forceinline__ static void store_a(void* A, int o, float nx, float ny, float nz, float d) {
    reinterpret_cast<float4*>(A)[o] = make_float4(nx, ny, nz, d);
  }
  __device__ __forceinline__ static void store_b(void* B, int o, float i, float gx, float gy, float d) {
    reinterpret_cast<float4*>(B)[o] = make_float4(i, gx, gy, d);
  }
  // normal and depth at pixel o (the depth plane D is not read)
  __device__ __forceinline__ static float4 load_a(const void* A, const float* D, int o) {
    return __ldg(reinterpret_cast<const float4*>(A) + o);
  }
  __device__ __forceinline__ static float depth(const void* A, const float* D, int o) {
    return __ldg(reinterpret_cast<const float*>(A) + 4 * o + 3);
  }
  // intensity, g_x, g_y (and the depth) at pixel o
  __device__ __forceinline__ static float4 load_b(const void* B, int o) {
    return __ldg(reinterpret_cast<const float4*>(B) + o);
  }
};

template <>
struct Packs<__half> {
  static constexpr int kBytesA = 8, kBytesB = 8;
  static constexpr bool kDepthInB = false;
  __device__ __forceinline__ static void store_a(void* A, int o, float nx, float ny, float nz, float d) {
    const __half2 xy = __floats2half2_rn(nx, ny), z0 = __floats2half2_rn(nz, 0.f);
    uint2 v;
    v.x = *reinterpret_cast<const unsigned int*>(&xy);
    v.y = *reinterpret_cast<const unsigned int*>(&z0);
    reinterpret_cast<uint2*>(A)[o] = v;
  }
  __device__ __forceinline__ static void store_b(void* B, int o, float i, float gx, float gy, float) {
    const __half2 g = __floats2half2_rn(gx, gy);
    uint2 v;
    v.x = __float_as_uint(i);
    v.y = *reinterpret_cast<const unsigned int*>(&g);
    reinterpret_cast<uint2*>(B)[o] = v;
  }
  __device__ __forceinline__ static float4 load_a(const void* A, const float* D, int o) {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(A) + o);
    const float2 xy = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
    const float2 z0 = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
    return make_float4(xy.x, xy.y, z0.x, __ldg(D + o));
  }
  __device__ __forceinline__ static float depth(const void* A, const float* D, int o) {
    return __ldg(D + o);
  }
  __device__ __forceinline__ static float4 load_b(const void* B, int o) {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(B) + o);
    const float2 g = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
    return make_float4(__uint_as_float(v.x), g.x, g.y, 0.f);
  }
};

}  // namespace dri
