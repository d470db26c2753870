// Fused per-pixel Gauss-Newton linearisation of the photometric (Eq. 3) and
// point-to-plane ICP (Eq. 4) terms at one pyramid level, block-reduced into the
// normal equations of Eq. 7 (Sec. IV-B, IV-D).
//
// A thread evaluates one term only and carries that term's 29 sums: half the
// registers of a thread that does both, more warps resident per SM to hide the
// latency of the dependent gathers.  Batched kernel: a block of 8 warps takes
// one term over a tile of 32 columns x 8 * ppt rows (warp w: rows w, w + 8, ...),
// the two terms of a tile being neighbouring blocks, so a block never waits at
// its final barrier for the other (slower) term.  By-value kernel (per-pixel
// flags of the allocation-free entry): warps 0-3 ICP and 4-7 photometric over
// the same 32 x 4 * ppt pixels.  Each gather is one vector load of a per-pixel
// pack (packs.cuh): the ICP term reads pack A (normal + depth) of the live pixel
// and of the associated reference pixel, the photometric term the live depth
// and intensity and four pack-B taps (intensity + gradient) of the reference.
// A pixel's work is a front half (the point, its projection, the tests that
// need no reference sample, the gather) and a back half (the tests on the
// reference sample, residual, Jacobian, sums); every test is a comparison that
// NaN fails, so no pixel branches away before its gather.  Each thread loads
// its next row's live samples before it works on the current one, and asks L2
// for the reference samples its next row is expected to gather.  Per pixel, in
// FP32:
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
// e^2, count) in FP32, 28 of them in pairs by packed FP32 x 2 FMAs (14 per
// pixel instead of 28 scalar ones); a warp transposes and sums them with 31 shuffles, the
// block adds its warps per term in fixed order into one FP64 (or FP32)
// partial of 58 values; the partials are folded in two fixed-order levels
// (groups of blocks, then the groups) into ctrl->sums: deterministic, no float
// atomics.
#include <cuda_fp16.h>

#include "dri_internal.h"
#include "packs.cuh"

namespace dri {

namespace {

// The 29 sums of a thread, stored in pairs for the packed FP32 x 2 FMA: slot
// acc_slot(k) holds sum k of the row-major upper J J^T (0..20), J e (21..26),
// e^2 (27), count (28).  Each pair is one fma.rn.f32x2 per pixel, each lane
// rounded as a scalar fmaf, so every sum is bit-identical to scalar accumulation.
__host__ __device__ constexpr int acc_slot(int k) {
  constexpr int pos[29] = {0, 18, 6, 8, 10, 12, 1, 9, 7, 13, 11, 2, 19, 14, 16,
                           3, 17, 15, 4, 20, 5, 22, 23, 24, 25, 26, 27, 21, 28};
  return pos[k];
}

__device__ __forceinline__ void fma2(float* a, float2 x, float2 y) {
  const float2 r = __ffma2_rn(x, y, make_float2(a[0], a[1]));
  a[0] = r.x;
  a[1] = r.y;
}

__device__ __forceinline__ void accumulate(float* a, const float* J, float e) {
  const float2 P0 = make_float2(J[0], J[1]), P1 = make_float2(J[2], J[3]), P2 = make_float2(J[4], J[5]);
  const float2 S1 = make_float2(J[3], J[2]), S2 = make_float2(J[5], J[4]);
  const float2 E = make_float2(e, e);
  fma2(a + 0, P0, P0);
  fma2(a + 2, P1, P1);
  fma2(a + 4, P2, P2);
  fma2(a + 6, P0, P1);
  fma2(a + 8, P0, S1);
  fma2(a + 10, P0, P2);
  fma2(a + 12, P0, S2);
  fma2(a + 14, P1, P2);
  fma2(a + 16, P1, S2);
  fma2(a + 18, make_float2(J[0], J[2]), make_float2(J[1], J[3]));
  fma2(a + 20, make_float2(J[4], e), make_float2(J[5], e));
  fma2(a + 22, P0, E);
  fma2(a + 24, P1, E);
  fma2(a + 26, P2, E);
  a[28] += 1.f;
}

// Rows ahead of the current one whose live samples each thread asks L2 to fetch
// (0: none).  The reference is prefetched where the thread's next row is
// expected to land: one thread row (kR image rows) below the current gather,
// which for a smooth surface and a small motion is where the next pixel
// projects (measured: long-scoreboard stalls 5.9 -> 4.2 per issued
// instruction, 69 -> 66 us per 16-slot launch).
constexpr int kPrefetchRows = 4;

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Margin decisions (the last iteration of each level, and the parity entry):
// a pixel whose accept / reject decision in this kernel lies within 1e-4 px of
// a rounding or bound boundary, or within a relative 1e-5 of a threshold, as
// the oracle marks its margin pixels; an FP32 and an FP64 evaluation may
// decide it differently.
constexpr float kPxMargin = 1e-4f, kRelMargin = 1e-5f;
__device__ __forceinline__ bool near_rel(float a, float thr) {
  return fabsf(a - thr) <= kRelMargin * fabsf(thr);
}
// f - floor(f) within kPxMargin of 0 or 1 (f's integer part is fl)
__device__ __forceinline__ bool near_int(float f, float fl) {
  const float r = f - fl;
  return r < kPxMargin || r > 1.f - kPxMargin;
}

// What a thread needs of its tile for the whole loop over its rows: the term's
// transform (A = R^T R_1 - I, t), its column u with the pixel ray's x part and
// the bounds of an integer displacement that stays inside the reference image,
// and the maps.
struct TileCtx {
  LevelGeom g;
  float A[9], t[3];
  int u;
  bool col_ok;
  float rx;                     // (u - c_x) / f_x
  float ucx;                    // u - c_x
  float lox, hix;               // -u and w - u: x + u in [0, w) <=> lox <= x < hix
  float ify_cy;                 // -c_y / f_y
  int row0, kR, nrows;          // the thread's rows: row0, row0 + kR, ... (nrows of them)
  float dmin, dmax, dist2, cosmin, occ_thr;
  float dist2_lo, dist2_hi;     // margin decisions: squared distances within 1e-5 of the threshold
  float cos_margin;             //   and the angle test's margin
  const void* __restrict__ A1;  // live pack A
  const float* __restrict__ D1;
  const float* __restrict__ I1;
  const void* __restrict__ A0;  // reference packs
  const float* __restrict__ D0;
  const void* __restrict__ B0;
  uint8_t* flags;
};

// Row constants of the thread's pixel (u, v).
struct RowCtx {
  int v, o;                     // row and pixel index v w + u
  bool in;                      // the pixel exists
  float ry;                     // (v - c_y) / f_y
  float vcy;                    // v - c_y
  float loy, hiy;               // -v and h - v
};

__device__ __forceinline__ RowCtx row_ctx(const TileCtx& c, int r) {
  RowCtx q;
  q.v = c.row0 + r * c.kR;
  q.o = q.v * c.g.w + c.u;
  q.in = c.col_ok && q.v < c.g.h;
  const float vf = (float)q.v;
  q.ry = fmaf(vf, c.g.ify, c.ify_cy);
  q.vcy = vf - c.g.cy;
  q.loy = -vf;
  q.hiy = (float)c.g.h - vf;
  return q;
}

// The live point p = d (r_x, r_y, 1) and D = A p + t: p + D is the point in the
// reference (ICP) or x0 (photometric) camera.
struct Warp3 {
  float px, py, d, Dx, Dy, Dz;
};

__device__ __forceinline__ Warp3 warp_point(const TileCtx& c, float ry, float d) {
  Warp3 w;
  w.px = d * c.rx;
  w.py = d * ry;
  w.d = d;
  w.Dx = fmaf(c.A[0], w.px, fmaf(c.A[1], w.py, fmaf(c.A[2], d, c.t[0])));
  w.Dy = fmaf(c.A[3], w.px, fmaf(c.A[4], w.py, fmaf(c.A[5], d, c.t[1])));
  w.Dz = fmaf(c.A[6], w.px, fmaf(c.A[7], w.py, fmaf(c.A[8], d, c.t[2])));
  return w;
}

// ---- ICP term (Eq. 4) -------------------------------------------------------
// Front half: association and the gather of the reference pack; back half:
// residual, Jacobian and accumulation.
struct IcpPix {
  float4 ref;                   // reference pack A at the associated pixel: N, d_ref
  Warp3 w;
  float ix, iy;                 // integer displacement of the associated pixel
  float mx, my, mz;             // (I + A) n1: the live normal in the reference camera
  bool ok;
  bool cand;                    // depth in range and a normal: the tests after the gather apply
  bool m;                       // a margin decision so far
};

template <typename T, bool MARGIN>
__device__ __forceinline__ void icp_front(const TileCtx& c, const RowCtx& q, const float4 live,
                                          IcpPix& x) {
  // live = (n1, d); a zero normal is rejected by the angle test (cos_min > 0)
  const float d = live.w;
  x.w = warp_point(c, q.ry, d);
  const float z = d + x.w.Dz;
  const float iz = __fdividef(1.f, z);
  // displacement of the projection from (u, v): small, so FP32 keeps it to
  // ~1e-5 px, and the integer parts of the position stay exact
  const float sx = c.g.fx * (fmaf(-c.rx, x.w.Dz, x.w.Dx) * iz);
  const float sy = c.g.fy * (fmaf(-q.ry, x.w.Dz, x.w.Dy) * iz);
  x.ix = floorf(sx + 0.5f);                    // nearest pixel
  x.iy = floorf(sy + 0.5f);
  // NaN and out-of-range displacements fail these comparisons
  x.ok = q.in && d >= c.dmin && d <= c.dmax && z > 0.f && x.ix >= c.lox && x.ix < c.hix &&
         x.iy >= q.loy && x.iy < q.hiy;
  if (MARGIN) {
    const bool dv = q.in && d >= c.dmin && d <= c.dmax;
    x.cand = dv && (live.x != 0.f || live.y != 0.f || live.z != 0.f);
    const float pz = d + x.w.Dz, px = x.w.px + x.w.Dx, py = x.w.py + x.w.Dy;
    // |z| <= 1e-5 |p| as squares (1e-10 = kRelMargin^2)
    x.m = (dv && (near_rel(d, c.dmin) || near_rel(d, c.dmax))) ||
          (x.cand && pz * pz <= 1e-10f * fmaf(px, px, fmaf(py, py, pz * pz))) ||
          (x.cand && pz > 0.f && (near_int(sx + 0.5f, x.ix) || near_int(sy + 0.5f, x.iy)));
  }
  x.mx = fmaf(c.A[0], live.x, fmaf(c.A[1], live.y, fmaf(c.A[2], live.z, live.x)));
  x.my = fmaf(c.A[3], live.x, fmaf(c.A[4], live.y, fmaf(c.A[5], live.z, live.y)));
  x.mz = fmaf(c.A[6], live.x, fmaf(c.A[7], live.y, fmaf(c.A[8], live.z, live.z)));
  x.ref = make_float4(0.f, 0.f, 0.f, 0.f);
  if (x.ok) {
    const int a = q.o + (int)x.iy * c.g.w + (int)x.ix;
    x.ref = Packs<T>::load_a(c.A0, c.D0, a);
    if (x.iy + (float)c.kR < q.hiy)          // the thread's next row, kR reference rows down
      prefetch_l2(static_cast<const char*>(c.A0) + (size_t)(a + c.kR * c.g.w) * Packs<T>::kBytesA);
  }
}

template <bool DW, bool FLAGS, bool MARGIN>
__device__ __forceinline__ void icp_back(const TileCtx& c, const RowCtx& q, const IcpPix& x,
                                         float* acc, int& nm) {
  const float Nx = x.ref.x, Ny = x.ref.y, Nz = x.ref.z, dr = x.ref.w;
  // reference vertex V = d_ref K^-1 [x_i, y_i, 1]^T
  const float Vx = dr * ((c.ucx + x.ix) * c.g.ifx);
  const float Vy = dr * ((q.vcy + x.iy) * c.g.ify);
  const float dx = (x.w.px - Vx) + x.w.Dx, dy = (x.w.py - Vy) + x.w.Dy, dz = (x.w.d - dr) + x.w.Dz;
  const float dist2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  const float cosang = fmaf(x.mx, Nx, fmaf(x.my, Ny, x.mz * Nz));
  const bool ok = x.ok && dist2 < c.dist2 && cosang > c.cosmin;
  bool m = false;
  if (MARGIN) {                // distance and angle tests at a valid reference pixel
    const bool rvalid = x.ok && (Nx != 0.f || Ny != 0.f || Nz != 0.f);   // a reference normal
    m = x.m || (x.cand && rvalid &&
                ((dist2 >= c.dist2_lo && dist2 <= c.dist2_hi) || fabsf(cosang - c.cosmin) <= c.cos_margin));
    nm += m ? 1 : 0;
  }
  if (FLAGS && (ok || m)) {    // bit 0 valid, the association in bits 2-5, bit 6 margin
    const unsigned xi = (unsigned)(c.u + (int)x.ix), yi = (unsigned)(q.v + (int)x.iy);
    const unsigned bits = (ok ? 1u | (xi & 3u) << 2 | (yi & 3u) << 4 : 0u) | (m ? 1u << 6 : 0u);
    atomicOr(reinterpret_cast<unsigned int*>(c.flags + (q.o & ~3)), bits << (8 * (q.o & 3)));
  }
  if (!ok) return;
  const float e = fmaf(Nx, dx, fmaf(Ny, dy, Nz * dz));
  // s = (I + A) p: the live point rotated into the reference camera
  const float sx = x.w.px + (x.w.Dx - c.t[0]), sy = x.w.py + (x.w.Dy - c.t[1]),
              sz = x.w.d + (x.w.Dz - c.t[2]);
  const float J[6] = {Nx, Ny, Nz, sy * Nz - sz * Ny, sz * Nx - sx * Nz, sx * Ny - sy * Nx};
  if (DW) {                      // weight 1 / d^4 (sigma_d(d) = sigma_d d^2): J, e scaled by 1 / d^2
    const float wgt = __fdividef(1.f, x.w.d * x.w.d);
    const float Jw[6] = {J[0] * wgt, J[1] * wgt, J[2] * wgt, J[3] * wgt, J[4] * wgt, J[5] * wgt};
    accumulate(acc, Jw, e * wgt);
    return;
  }
  accumulate(acc, J, e);
}

// ---- photometric term (Eq. 3) ------------------------------------------------
struct RgbPix {
  float4 s00, s01, s10, s11;    // reference pack B at the four bilinear taps
  Warp3 w;
  float ax, ay;                 // bilinear weights of the right / lower taps
  float xr, yr;                 // x - c_x, y - c_y of the warped point
  float iz, z;
  float i1;                     // live intensity
  bool ok;
  bool m;                       // a margin decision so far
};

template <typename T, bool MARGIN>
__device__ __forceinline__ void rgb_front(const TileCtx& c, const RowCtx& q, float d, float i1,
                                          RgbPix& x) {
  x.w = warp_point(c, q.ry, d);
  x.z = d + x.w.Dz;
  x.iz = __fdividef(1.f, x.z);
  const float sx = c.g.fx * (fmaf(-c.rx, x.w.Dz, x.w.Dx) * x.iz);
  const float sy = c.g.fy * (fmaf(-q.ry, x.w.Dz, x.w.Dy) * x.iz);
  const float fx = floorf(sx), fy = floorf(sy);
  // the bilinear support [x, x + 1] x [y, y + 1] inside the image
  x.ok = q.in && d >= c.dmin && d <= c.dmax && x.z > 0.f && fx >= c.lox && fx < c.hix - 1.f &&
         fy >= q.loy && fy < q.hiy - 1.f;
  if (MARGIN) {
    const bool dv = q.in && d >= c.dmin && d <= c.dmax;
    const float px = x.w.px + x.w.Dx, py = x.w.py + x.w.Dy;
    // x = u + sx, so |x| = |sx - lox| and |x - (w - 1)| = |sx - (hix - 1)|
    x.m = (dv && (near_rel(d, c.dmin) || near_rel(d, c.dmax))) ||
          (dv && x.z * x.z <= 1e-10f * fmaf(px, px, fmaf(py, py, x.z * x.z))) ||
          (dv && x.z > 0.f &&
           (fabsf(sx - c.lox) <= kPxMargin || fabsf(sx - (c.hix - 1.f)) <= kPxMargin ||
            fabsf(sy - q.loy) <= kPxMargin || fabsf(sy - (q.hiy - 1.f)) <= kPxMargin));
  }
  x.ax = sx - fx;
  x.ay = sy - fy;
  x.xr = c.ucx + sx;
  x.yr = q.vcy + sy;
  x.i1 = i1;
  x.s00 = x.s01 = x.s10 = x.s11 = make_float4(0.f, 0.f, 0.f, 0.f);
  if (x.ok) {
    const int b = q.o + (int)fy * c.g.w + (int)fx;
    x.s00 = Packs<T>::load_b(c.B0, b);
    x.s01 = Packs<T>::load_b(c.B0, b + 1);
    x.s10 = Packs<T>::load_b(c.B0, b + c.g.w);
    x.s11 = Packs<T>::load_b(c.B0, b + c.g.w + 1);
    if (fy + (float)(c.kR + 1) < q.hiy) {    // the next row's two tap rows, kR rows down
      const char* B = static_cast<const char*>(c.B0);
      prefetch_l2(B + (size_t)(b + c.kR * c.g.w) * Packs<T>::kBytesB);
      prefetch_l2(B + (size_t)(b + (c.kR + 1) * c.g.w) * Packs<T>::kBytesB);
    }
  }
}

template <typename T, bool OCC, bool FLAGS, bool MARGIN>
__device__ __forceinline__ void rgb_back(const TileCtx& c, const RowCtx& q, const RgbPix& x,
                                         float* acc, int& nm) {
  bool ok = x.ok;
  bool m = MARGIN && x.m;
  if (OCC && ok) {               // depth consistency at the nearest reference pixel
    const bool right = x.ax >= 0.5f, down = x.ay >= 0.5f;
    float dr;
    if (Packs<T>::kDepthInB) {
      dr = down ? (right ? x.s11.w : x.s10.w) : (right ? x.s01.w : x.s00.w);
    } else {
      const float sx = x.xr - c.ucx, sy = x.yr - q.vcy;
      dr = __ldg(c.D0 + q.o + (int)(floorf(sy) + (down ? 1.f : 0.f)) * c.g.w +
                 (int)(floorf(sx) + (right ? 1.f : 0.f)));
    }
    if (MARGIN)                  // the nearest pixel's rounding and the depth gap's threshold
      m = m || fabsf(x.ax - 0.5f) < kPxMargin || fabsf(x.ay - 0.5f) < kPxMargin ||
          (dr > 0.f && near_rel(fabsf(x.z - dr), c.occ_thr));
    if (dr > 0.f && fabsf(x.z - dr) > c.occ_thr) ok = false;
  }
  if (MARGIN) nm += m ? 1 : 0;
  if (FLAGS && (ok || m))        // bit 1 valid, bit 7 margin
    atomicOr(reinterpret_cast<unsigned int*>(c.flags + (q.o & ~3)),
             ((ok ? 2u : 0u) | (m ? 1u << 7 : 0u)) << (8 * (q.o & 3)));
  if (!ok) return;
  const float w00 = (1.f - x.ax) * (1.f - x.ay), w01 = x.ax * (1.f - x.ay);
  const float w10 = (1.f - x.ax) * x.ay, w11 = x.ax * x.ay;
  const float iv = w00 * x.s00.x + w01 * x.s01.x + w10 * x.s10.x + w11 * x.s11.x;
  const float gx = w00 * x.s00.y + w01 * x.s01.y + w10 * x.s10.y + w11 * x.s11.y;
  const float gy = w00 * x.s00.z + w01 * x.s01.z + w10 * x.s10.z + w11 * x.s11.z;
  const float e = iv - x.i1;
  const float a0 = c.g.fx * gx * x.iz, a1 = c.g.fy * gy * x.iz;
  const float a2 = -(gx * x.xr + gy * x.yr) * x.iz;
  const float sx = x.w.px + (x.w.Dx - c.t[0]), sy = x.w.py + (x.w.Dy - c.t[1]),
              sz = x.w.d + (x.w.Dz - c.t[2]);
  const float J[6] = {a0, a1, a2, sy * a2 - sz * a1, sz * a0 - sx * a2, sx * a1 - sy * a0};
  accumulate(acc, J, e);
}

// L2 prefetch of the live samples kPrefetchRows rows ahead.
template <typename T>
__device__ __forceinline__ void prefetch_ahead(const TileCtx& c, int r, bool icp) {
  if (kPrefetchRows <= 0 || r + kPrefetchRows >= c.nrows) return;
  const int v = c.row0 + (r + kPrefetchRows) * c.kR;
  if (!c.col_ok || v >= c.g.h) return;
  const int o = v * c.g.w + c.u;
  if (icp) prefetch_l2(static_cast<const char*>(c.A1) + (size_t)o * Packs<T>::kBytesA);
  else prefetch_l2(c.I1 + o);
}

// The ICP term over the thread's rows: each row's live pack is loaded one row
// ahead; its front half (association, reference gather) and back half
// (residual, Jacobian, sums) follow each other.  (Issuing the next row's front
// half before the current row's back half, so that its gather is in flight
// meanwhile, measured slower: the state carried between the halves costs
// registers -- fewer resident warps or spills -- and moves.)
template <typename T, bool DW, bool FLAGS, bool MARGIN>
__device__ __forceinline__ void icp_rows(const TileCtx& c, float* acc, int& nm) {
  auto live = [&](const RowCtx& q) {
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
    if (q.in) a = Packs<T>::load_a(c.A1, c.D1, q.o);
    return a;
  };
  float4 l = live(row_ctx(c, 0));
  for (int r = 0; r < c.nrows; ++r) {
    const RowCtx q = row_ctx(c, r);
    const float4 ln = r + 1 < c.nrows ? live(row_ctx(c, r + 1)) : make_float4(0.f, 0.f, 0.f, 0.f);
    prefetch_ahead<T>(c, r, true);
    IcpPix x;
    icp_front<T, MARGIN>(c, q, l, x);
    icp_back<DW, FLAGS, MARGIN>(c, q, x, acc, nm);
    l = ln;
  }
}

// The photometric term over the thread's rows, as icp_rows.
template <typename T, bool OCC, bool FLAGS, bool MARGIN>
__device__ __forceinline__ void rgb_rows(const TileCtx& c, float* acc, int& nm) {
  auto live = [&](const RowCtx& q) {
    float2 a = make_float2(0.f, 0.f);
    if (q.in) a = make_float2(Packs<T>::depth(c.A1, c.D1, q.o), __ldg(c.I1 + q.o));
    return a;
  };
  float2 l = live(row_ctx(c, 0));
  for (int r = 0; r < c.nrows; ++r) {
    const RowCtx q = row_ctx(c, r);
    const float2 ln = r + 1 < c.nrows ? live(row_ctx(c, r + 1)) : make_float2(0.f, 0.f);
    prefetch_ahead<T>(c, r, false);
    RgbPix x;
    rgb_front<T, MARGIN>(c, q, l.x, l.y, x);
    rgb_back<T, OCC, FLAGS, MARGIN>(c, q, x, acc, nm);
    l = ln;
  }
}

// One tile of one image (single-term: 32 x 8 * ppt pixels of `term`; mixed:
// 32 x 4 * ppt pixels, warps 0-3 ICP and 4-7 photometric): (bx, by) its tile
// coordinates, bid its index in the image's fold order.
// Optional terms, compile-time variants of the pixel kernels (OPT bits): the
// photometric occlusion test and the depth-dependent ICP weight.
constexpr int kOptOcc = 1, kOptDepthWeight = 2;

template <typename T, typename P, bool FLAGS, bool MARGIN, bool SPLIT, int OPT>
__device__ __forceinline__ void track_tile(const TrackParams& p, const int term, const int bx,
                                           const int by, const int bid) {
  Ctrl* __restrict__ ctrl = p.ctrl;
  if (ctrl->status != 0) return;
  const int lane = threadIdx.x;
  const int warp = threadIdx.y;
  const bool icp = SPLIT ? term == 0 : warp < kTrackRows;    // warp-uniform
  const int wrow = SPLIT ? warp : (warp & (kTrackRows - 1));
  const int rs = ctrl->ref_index;
  const int cs = 1 - rs;

  TileCtx c;
  c.g = p.g;
  const float* xf = icp ? ctrl->xf_icp : ctrl->xf_rgb;
#pragma unroll
  for (int k = 0; k < 9; ++k) c.A[k] = xf[k];
#pragma unroll
  for (int k = 0; k < 3; ++k) c.t[k] = xf[9 + k];
  c.u = bx * kTrackThreadsX + lane;
  c.col_ok = c.u < c.g.w;
  const float uf = (float)c.u;
  c.rx = (uf - c.g.cx) * c.g.ifx;
  c.ucx = uf - c.g.cx;
  c.lox = -uf;
  c.hix = (float)c.g.w - uf;
  c.ify_cy = -c.g.cy * c.g.ify;
  c.kR = SPLIT ? kTrackThreadsY : kTrackRows;                // rows between a thread's rows
  c.row0 = by * p.ppt * c.kR + wrow;
  c.nrows = p.ppt;
  c.dmin = p.depth_min;
  c.dmax = p.depth_max;
  c.dist2 = p.icp_dist2;
  c.cosmin = p.icp_cos;
  {
    const float thr = sqrtf(p.icp_dist2);
    c.dist2_lo = (thr * (1.f - kRelMargin)) * (thr * (1.f - kRelMargin));
    c.dist2_hi = (thr * (1.f + kRelMargin)) * (thr * (1.f + kRelMargin));
  }
  // FP16 normals: a stored normal may be one half-precision unit from the
  // rounding of an FP64-computed one, which moves cos by up to ~2 * 2^-11
  c.cos_margin = sizeof(T) == 2 ? 4.f * 0.00048828125f : kRelMargin * fabsf(p.icp_cos);
  c.occ_thr = p.occ_thr;
  c.A1 = p.m.packA[cs];
  c.D1 = p.m.depth[cs];
  c.I1 = p.m.inten[cs];
  c.A0 = p.m.packA[rs];
  c.D0 = p.m.depth[rs];
  c.B0 = p.m.packB[rs];
  c.flags = p.flags;

  float acc[kSums];
#pragma unroll
  for (int k = 0; k < kSums; ++k) acc[k] = 0.f;
  int nm = 0;
  if (icp) icp_rows<T, (OPT & kOptDepthWeight) != 0, FLAGS, MARGIN>(c, acc, nm);
  else rgb_rows<T, (OPT & kOptOcc) != 0, FLAGS, MARGIN>(c, acc, nm);
  if (MARGIN) {                      // the warp's margin decisions, one integer add
    const unsigned sum = __reduce_add_sync(0xffffffffu, (unsigned)nm);
    if (lane == 0 && sum) atomicAdd(&ctrl->margin_acc[icp ? 0 : 1], sum);
  }

  // ---------------- reduction ----------------
  // Warp: transpose-reduce.  Padded to 32 values, five halving exchanges leave
  // lane l holding the warp sum of value l (31 shuffles instead of 5 per value).
  float w[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) w[k] = k < kSums ? acc[acc_slot(k)] : 0.f;
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
  track_tile<T, P, FLAGS, FLAGS, false, OPT>(p, 0, blockIdx.x, blockIdx.y, blockIdx.y * gridDim.x + blockIdx.x);
}

// Tiles of every tracking slot at one level: block -> (slot, tile, term)
// through the block prefix, tile -> (column, row band) in the slot's image.
// Three blocks per SM (80 registers) measured faster than four (64 registers,
// more spill reloads) and than two columns per thread.
// FLAGS (parity entry only): the same kernel that also or-s each pixel's
// validity bits into a.flags (the slot's level image, zeroed before the launch).
template <typename T, typename P, int OPT, bool FLAGS, bool MARGIN>
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
  track_tile<T, P, FLAGS, MARGIN, true, OPT>(p, t & 1, tile % gx, tile / gx, t);
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
#define DRI_TRACK_BATCH_F(T, P, F, M)                                                    \
  do {                                                                                   \
    if (opt == 0) return cudaLaunchKernelEx(&cfg, k_track_batch<T, P, 0, F, M>, a);      \
    if (opt == 1) return cudaLaunchKernelEx(&cfg, k_track_batch<T, P, 1, F, M>, a);      \
    if (opt == 2) return cudaLaunchKernelEx(&cfg, k_track_batch<T, P, 2, F, M>, a);      \
    return cudaLaunchKernelEx(&cfg, k_track_batch<T, P, 3, F, M>, a);                    \
  } while (0)
#define DRI_TRACK_BATCH(T, P)                                                            \
  do {                                                                                   \
    if (a.flags) DRI_TRACK_BATCH_F(T, P, true, true);                                    \
    if (a.margin) DRI_TRACK_BATCH_F(T, P, false, true);                                  \
    DRI_TRACK_BATCH_F(T, P, false, false);                                               \
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
