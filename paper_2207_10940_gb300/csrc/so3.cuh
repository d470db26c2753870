// FP64 rotation algebra for the solver kernels (Sec. II conventions, Eq. 2).
// Hamilton quaternions (w, x, y, z); 3x3 matrices row-major; global (left)
// perturbations q <- exp(da) (x) q.
#pragma once

#include <cuda_runtime.h>

namespace dri {

// Below this theta^2 (theta < 0.05 rad) the rotation functions use their Taylor
// series in theta^2 (five terms, relative error below 1e-16 there): on this GPU a
// dependent FP64 FMA costs ~64 cycles but a sincos ~1.4k and a sqrt or divide
// several hundred, and most angles here (IMU pieces, residuals, GN steps) are small.
constexpr double kSeriesT2 = 2.5e-3;

__device__ __forceinline__ void m3_mul(const double* A, const double* B, double* C) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}

// C = A^T B
__device__ __forceinline__ void m3_tmul(const double* A, const double* B, double* C) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      C[3 * i + j] = A[i] * B[j] + A[3 + i] * B[3 + j] + A[6 + i] * B[6 + j];
}

// C = A B^T
__device__ __forceinline__ void m3_mult(const double* A, const double* B, double* C) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      C[3 * i + j] = A[3 * i] * B[3 * j] + A[3 * i + 1] * B[3 * j + 1] + A[3 * i + 2] * B[3 * j + 2];
}

__device__ __forceinline__ void m3_vec(const double* A, const double* x, double* y) {
#pragma unroll
  for (int i = 0; i < 3; ++i) y[i] = A[3 * i] * x[0] + A[3 * i + 1] * x[1] + A[3 * i + 2] * x[2];
}

__device__ __forceinline__ void m3_tvec(const double* A, const double* x, double* y) {
#pragma unroll
  for (int i = 0; i < 3; ++i) y[i] = A[i] * x[0] + A[3 + i] * x[1] + A[6 + i] * x[2];
}

__device__ __forceinline__ void hat3(const double* w, double* K) {
  K[0] = 0.0;   K[1] = -w[2]; K[2] = w[1];
  K[3] = w[2];  K[4] = 0.0;   K[5] = -w[0];
  K[6] = -w[1]; K[7] = w[0];  K[8] = 0.0;
}

__device__ __forceinline__ void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

// I + a K + b K^2 with K = hat(w)
__device__ __forceinline__ void rodrigues_form(const double* w, double a, double b, double* R) {
  const double x = w[0], y = w[1], z = w[2];
  // K^2 = w w^T - |w|^2 I
  const double n2 = x * x + y * y + z * z;
  R[0] = 1.0 + b * (x * x - n2); R[1] = -a * z + b * x * y;   R[2] = a * y + b * x * z;
  R[3] = a * z + b * x * y;      R[4] = 1.0 + b * (y * y - n2); R[5] = -a * x + b * y * z;
  R[6] = -a * y + b * x * z;     R[7] = a * x + b * y * z;      R[8] = 1.0 + b * (z * z - n2);
}

// Exp of a rotation vector (Rodrigues): I + sin(t)/t K + (1 - cos t)/t^2 K^2.
__device__ __forceinline__ void so3_exp(const double* w, double* R) {
  const double t2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double a, b;
  if (t2 < kSeriesT2) {
    a = 1.0 + t2 * (-1.0 / 6 + t2 * (1.0 / 120 + t2 * (-1.0 / 5040 + t2 * (1.0 / 362880))));
    b = 0.5 + t2 * (-1.0 / 24 + t2 * (1.0 / 720 + t2 * (-1.0 / 40320 + t2 * (1.0 / 3628800))));
  } else {
    const double t = sqrt(t2);
    double s, c;
    sincos(t, &s, &c);
    a = s / t;
    b = (1.0 - c) / t2;
  }
  rodrigues_form(w, a, b, R);
}

// Right Jacobian Jr(w) = I - (1 - cos t)/t^2 K + (t - sin t)/t^3 K^2:
// Exp(w + d) ~= Exp(w) Exp(Jr d).
__device__ __forceinline__ void so3_jr(const double* w, double* J) {
  const double t2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double a, b;
  if (t2 < kSeriesT2) {
    a = 0.5 + t2 * (-1.0 / 24 + t2 * (1.0 / 720 + t2 * (-1.0 / 40320 + t2 * (1.0 / 3628800))));
    b = 1.0 / 6 + t2 * (-1.0 / 120 + t2 * (1.0 / 5040 + t2 * (-1.0 / 362880 + t2 * (1.0 / 39916800))));
  } else {
    const double t = sqrt(t2);
    double s, c;
    sincos(t, &s, &c);
    a = (1.0 - c) / t2;
    b = (t - s) / (t2 * t);
  }
  rodrigues_form(w, -a, b, J);
}

// Inverse left Jacobian: Log(Exp(d) Exp(w)) ~= w + Jl^-1(w) d, with
// Jl^-1 = I - K/2 + (1/t^2 - (1 + cos t)/(2 t sin t)) K^2.  Jr^-1(w) = Jl^-1(-w).
__device__ __forceinline__ void so3_jl_inv(const double* w, double* J) {
  const double t2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double c;
  if (t2 < kSeriesT2) {
    c = 1.0 / 12 + t2 * (1.0 / 720 + t2 * (1.0 / 30240 + t2 * (1.0 / 1209600 + t2 * (1.0 / 47900160))));
  } else {
    const double t = sqrt(t2);
    double s, co;
    sincos(t, &s, &co);
    c = 1.0 / t2 - (1.0 + co) / (2.0 * t * s);
  }
  rodrigues_form(w, -0.5, c, J);
}

__device__ __forceinline__ void so3_jr_inv(const double* w, double* J) {
  const double m[3] = {-w[0], -w[1], -w[2]};
  so3_jl_inv(m, J);
}

// Log of a rotation matrix (angle below pi - 1e-6).  The skew part is
// v = 2 sin(t) k; for small angles t / (2 sin t) = asin(s) / (2 s), s = sin t,
// is taken from its series in s^2 = |v|^2 / 4.
__device__ __forceinline__ void so3_log(const double* R, double* w) {
  const double c = 0.5 * (R[0] + R[4] + R[8] - 1.0);
  const double v0 = R[7] - R[5], v1 = R[2] - R[6], v2 = R[3] - R[1];
  double f;
  if (c > 0.99875) {                                  // t < 0.05
    const double s2 = 0.25 * (v0 * v0 + v1 * v1 + v2 * v2);
    f = 0.5 * (1.0 + s2 * (1.0 / 6 + s2 * (3.0 / 40 + s2 * (5.0 / 112 + s2 * (35.0 / 1152 +
               s2 * (63.0 / 2816 + s2 * (231.0 / 13312)))))));
  } else {
    const double t = acos(fmin(1.0, fmax(-1.0, c)));
    f = t / (2.0 * sin(t));
  }
  w[0] = f * v0;
  w[1] = f * v1;
  w[2] = f * v2;
}

// Rotation matrix of a unit quaternion (every quaternion stored here is kept unit).
__device__ __forceinline__ void quat_to_rot(const double* q, double* R) {
  const double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

__device__ __forceinline__ void quat_mul(const double* p, const double* q, double* o) {
  o[0] = p[0] * q[0] - p[1] * q[1] - p[2] * q[2] - p[3] * q[3];
  o[1] = p[0] * q[1] + p[1] * q[0] + p[2] * q[3] - p[3] * q[2];
  o[2] = p[0] * q[2] - p[1] * q[3] + p[2] * q[0] + p[3] * q[1];
  o[3] = p[0] * q[3] + p[1] * q[2] - p[2] * q[1] + p[3] * q[0];
}

// exp of a rotation vector as a unit quaternion: (cos(t/2), sin(t/2)/t w).
__device__ __forceinline__ void quat_exp(const double* w, double* q) {
  const double t2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double s, c;
  if (t2 < kSeriesT2) {
    s = 0.5 + t2 * (-1.0 / 48 + t2 * (1.0 / 3840 + t2 * (-1.0 / 645120 + t2 * (1.0 / 185794560))));
    c = 1.0 + t2 * (-1.0 / 8 + t2 * (1.0 / 384 + t2 * (-1.0 / 46080 + t2 * (1.0 / 10321920))));
  } else {
    const double t = sqrt(t2);
    double sh, ch;
    sincos(0.5 * t, &sh, &ch);
    s = sh / t;
    c = ch;
  }
  q[0] = c;
  q[1] = s * w[0];
  q[2] = s * w[1];
  q[3] = s * w[2];
}

// Renormalise a quaternion that is unit up to rounding: one Newton step of
// 1/sqrt(n2) about n2 = 1 (exact to O((n2 - 1)^2)); far from unit, a full rsqrt.
__device__ __forceinline__ void quat_normalise(double* q) {
  const double n2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
  const double f = fabs(n2 - 1.0) < 1e-6 ? 1.5 - 0.5 * n2 : rsqrt(n2);
#pragma unroll
  for (int i = 0; i < 4; ++i) q[i] *= f;
}

// Rotation of a unit quaternion from its matrix through the matrix log.
__device__ __forceinline__ void rot_to_quat(const double* R, double* q) {
  double w[3];
  so3_log(R, w);
  quat_exp(w, q);
}

// q <- exp(d) (x) q, normalised (Eq. 2)
__device__ __forceinline__ void quat_boxplus(double* q, const double* d) {
  double e[4], o[4];
  quat_exp(d, e);
  quat_mul(e, q, o);
  quat_normalise(o);
#pragma unroll
  for (int i = 0; i < 4; ++i) q[i] = o[i];
}

}  // namespace dri
