// FP64 rotation algebra for the solver kernels (Sec. II conventions, Eq. 2).
// Hamilton quaternions (w, x, y, z); 3x3 matrices row-major; global (left)
// perturbations q <- exp(da) (x) q.
#pragma once

#include <cuda_runtime.h>

namespace dri {

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

// Exp of a rotation vector (Rodrigues); series below 1e-3 rad.
__device__ __forceinline__ void so3_exp(const double* w, double* R) {
  const double t2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double a, b;
  if (t2 < 1e-6) {
    a = 1.0 - t2 / 6.0 + t2 * t2 / 120.0;
    b = 0.5 - t2 / 24.0 + t2 * t2 / 720.0;
  } else {
    const double t = sqrt(t2);
    double s, c;
    sincos(t, &s, &c);
    a = s / t;
    b = (1.0 - c) / t2;
  }
  rodrigues_form(w, a, b, R);
}

// Right Jacobian Jr(w): Exp(w + d) ~= Exp(w) Exp(Jr d).
__device__ __forceinline__ void so3_jr(const double* w, double* J) {
  const double t2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double a, b;
  if (t2 < 1e-6) {
    a = 0.5 - t2 / 24.0 + t2 * t2 / 720.0;
    b = 1.0 / 6.0 - t2 / 120.0 + t2 * t2 / 5040.0;
  } else {
    const double t = sqrt(t2);
    double s, c;
    sincos(t, &s, &c);
    a = (1.0 - c) / t2;
    b = (t - s) / (t2 * t);
  }
  rodrigues_form(w, -a, b, J);
}

// Inverse left Jacobian: Log(Exp(d) Exp(w)) ~= w + Jl^-1(w) d.  Jr^-1(w) = Jl^-1(-w).
__device__ __forceinline__ void so3_jl_inv(const double* w, double* J) {
  const double t2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double c;
  if (t2 < 1e-6) {
    c = 1.0 / 12.0 + t2 / 720.0 + t2 * t2 / 30240.0;
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

// Log of a rotation matrix (angle below pi - 1e-6).
__device__ __forceinline__ void so3_log(const double* R, double* w) {
  double c = 0.5 * (R[0] + R[4] + R[8] - 1.0);
  c = fmin(1.0, fmax(-1.0, c));
  const double t = acos(c);
  const double v0 = R[7] - R[5], v1 = R[2] - R[6], v2 = R[3] - R[1];
  double f;
  if (t < 1e-3) {
    f = 0.5 * (1.0 + t * t / 6.0 + 7.0 * t * t * t * t / 360.0);
  } else {
    f = t / (2.0 * sin(t));
  }
  w[0] = f * v0;
  w[1] = f * v1;
  w[2] = f * v2;
}

__device__ __forceinline__ void quat_to_rot(const double* qin, double* R) {
  const double n = rsqrt(qin[0] * qin[0] + qin[1] * qin[1] + qin[2] * qin[2] + qin[3] * qin[3]);
  const double w = qin[0] * n, x = qin[1] * n, y = qin[2] * n, z = qin[3] * n;
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

__device__ __forceinline__ void quat_exp(const double* w, double* q) {
  const double t2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double s, c;
  if (t2 < 1e-6) {
    s = 0.5 - t2 / 48.0 + t2 * t2 / 3840.0;
    c = 1.0 - t2 / 8.0 + t2 * t2 / 384.0;
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

__device__ __forceinline__ void quat_normalise(double* q) {
  const double n = rsqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
#pragma unroll
  for (int i = 0; i < 4; ++i) q[i] *= n;
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
