// FP64 single-block solver kernels of the tracking loop (Sec. IV-C/D/E).
//
//   frame_begin   x0 := x; IMU pre-integration at x0's biases with the propagated
//                 noise covariance; W_IMU = Sigma^-1; x1 := the IMU prediction x^1(x0)
//   gn_step       one Gauss-Newton iteration: re-integrate the IMU at x0's current
//                 biases, IMU error (Eq. 5) and its analytic 18x34 Jacobian; rotate
//                 the pixel kernel's photometric / ICP systems into W and map the
//                 photometric one onto both poses; add the prior (Eq. 6/9); solve the
//                 34x34 system of Eq. 7; x0, x1 boxplus= dx (Eq. 2)
//   frame_end     marginalise x0 by the Schur complement (Eq. 8) at the updated point,
//                 make the frame the reference (flip of the map sets)
//   frame_init    first frame (run by the frame-end kernel): first-frame prior, the
//                 frame becomes the reference
//
// Readings (the paper gives no integration scheme, Jacobians or prior sign):
// zero-order-hold integration cut at sample times, update order p, v, R; the bias
// Jacobians are the exact derivatives of that recursion; W_IMU is block diagonal
// (propagated (r, a, v) block, bias random walks, gravity noise) and fixed per
// frame; the prior adds H* to H_00 and b* - H* (x0 boxminus xbar) to b_0; after the
// last update b <- b - H dx before the Schur complement.
//
// GB300 design.  FP64 issue rate per SM is low, so the serial recursions are
// restated as data-parallel sums.  With dR_k the pre-integrated rotation before
// piece k (a prefix product, the only serial chain), u_k = dR_k (a_k - b_a),
// w_k = dt_k s_k + dt_k^2 / 2 (s_k = time left after piece k) and
// Y_k = dR_{k+1} Jr(theta_k):
//   dv = sum u_k dt_k,  dp = sum u_k w_k,
//   Psi_k = -sum_{i<k} Y_i dt_i,  d(dR)/d(b_g) = dR_N^T Psi_N,
//   d(dv, dp)/d(b_g) = -sum [u_k]x Psi_k (dt_k, w_k),  d(dv, dp)/d(b_a) = -sum dR_k (dt_k, w_k),
// and the noise covariance is the sum over pieces of each piece's noise carried
// to the end of the interval (state-transition blocks from suffix sums of u_k dt_k
// and u_k w_k).  These equal the sequential recursion exactly (same algebra,
// other rounding order).  W_IMU's block structure (a 9x9 block and a diagonal)
// is used in the assembly.  The step solves the reduced 26-dimensional system
// (x1's biases and gravity eliminated in closed form) with an element-parallel
// LDL^T on four warps; its 14 components that no pixel term touches are
// eliminated before the pixel sums arrive, the 12 pose components after
// (gn_step_body).  The 3-D gravity form solves its whole 36-dimensional system.
//
// All arithmetic here is FP64.  One block of kSolveThreads threads runs each
// stream's kernel; a batched launch has one block per slot.
#include <cmath>

#include "dri_internal.h"
#include "so3.cuh"

namespace dri {

namespace {

constexpr int kSolveThreads = 256;
constexpr int kMaxPieces = 128;

// ---------------------------------------------------------------------------
// IMU pieces and parallel pre-integration
// ---------------------------------------------------------------------------

__device__ __forceinline__ const dri_imu_sample* imu_samples(const ImuHeader* h) {
  return reinterpret_cast<const dri_imu_sample*>(h + 1);
}

// ---- element-wise 3x3 algebra: one output element per lane ----
// element e of op(A) op(B) (row-major; ta / tb transpose A / B)
__device__ __forceinline__ double mm_e(const double* A, const double* B, int e, bool ta, bool tb) {
  const int r = e / 3, c = e % 3;
  double v = 0.0;
#pragma unroll
  for (int k = 0; k < 3; ++k) v = fma(ta ? A[3 * k + r] : A[3 * r + k], tb ? B[3 * c + k] : B[3 * k + c], v);
  return v;
}
// element i of op(A) x
__device__ __forceinline__ double mv_e(const double* A, const double* x, int i, bool ta) {
  double v = 0.0;
#pragma unroll
  for (int k = 0; k < 3; ++k) v = fma(ta ? A[3 * k + i] : A[3 * i + k], x[k], v);
  return v;
}
// element e of [u]x
__device__ __forceinline__ double hat_e(const double* u, int e) {
  const int r = e / 3, c = e % 3;
  if (r == c) return 0.0;
  const double w = u[3 - r - c];
  return (((c - r + 3) % 3) == 1) ? -w : w;
}
// element e of [u]x M: (u x column c of M)_r
__device__ __forceinline__ double hatm_e(const double* u, const double* M, int e) {
  const int r = e / 3, c = e % 3, r1 = (r + 1) % 3, r2 = (r + 2) % 3;
  return u[r1] * M[3 * r2 + c] - u[r2] * M[3 * r1 + c];
}
// element e of op(M) [w]x: (row r of op(M) x w)_c
__device__ __forceinline__ double mhat_e(const double* M, bool tm, const double* w, int e) {
  const int r = e / 3, c = e % 3, c1 = (c + 1) % 3, c2 = (c + 2) % 3;
  const double m1 = tm ? M[3 * c1 + r] : M[3 * r + c1];
  const double m2 = tm ? M[3 * c2 + r] : M[3 * r + c2];
  return m1 * w[c2] - m2 * w[c1];
}

struct Preint {
  double dR[9], dv[3], dp[3];
  double Phig[9], Vg[9], Pg[9], Va[9], Pa[9];
  double Sig[81];                     // covariance of (dphi, dv, dp)
  double T;
};

struct ImuWork {
  double dR[kMaxPieces + 1][9];       // rotation before piece k
  double EP[kMaxPieces + 1][9];       // Exp(theta_k), then Psi_k
  double Y[kMaxPieces][9];            // Jr(theta_k), then dR_{k+1} Jr(theta_k)
  double u[kMaxPieces][3];            // a_k - b_a, then dR_k (a_k - b_a)
  double dt[kMaxPieces];
  double tau[kMaxPieces + 1];         // start of piece k relative to t0
  double w[kMaxPieces];
  double Cv[kMaxPieces + 1][3];       // suffix sums of u_k dt_k
  double Dv[kMaxPieces + 1][3];       // suffix sums of u_k w_k
  double ts[kMaxPieces + 2];          // sample times
  double S2[kMaxPieces][9];           // scan scratch
  int pk[kMaxPieces];
  int wcount[kSolveThreads / 32];     // valid pieces per warp (compaction)
  int np;
};

// Row r (0..8, order phi, v, p) of piece k's gyro-noise gain to the end of the
// interval, divided by dt_k.
__device__ __forceinline__ void gyro_gain_row(const ImuWork& W, int np, int k, int r, double* o) {
  const double* Yp = W.Y[k];
  if (r < 3) {
    const double* R = W.dR[np];
#pragma unroll
    for (int m = 0; m < 3; ++m) o[m] = R[r] * Yp[m] + R[3 + r] * Yp[3 + m] + R[6 + r] * Yp[6 + m];
  } else {
    const double* v = (r < 6 ? W.Cv : W.Dv)[k + 1];
    const int rr = r % 3;
    double h0, h1, h2;   // row rr of [v]x
    if (rr == 0) { h0 = 0.0; h1 = -v[2]; h2 = v[1]; }
    else if (rr == 1) { h0 = v[2]; h1 = 0.0; h2 = -v[0]; }
    else { h0 = -v[1]; h1 = v[0]; h2 = 0.0; }
#pragma unroll
    for (int m = 0; m < 3; ++m) o[m] = -(h0 * Yp[m] + h1 * Yp[3 + m] + h2 * Yp[6 + m]);
  }
}

// Whole block.  Pre-integration at biases (bg, ba) into P (and the noise
// covariance when cov).  Returns false (for all threads) if the samples do not
// cover the interval.
__device__ bool preintegrate_block(const ImuHeader* h, const double* bg, const double* ba, bool cov,
                                   double gnd, double and_, ImuWork& W, Preint& P) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31;
  const dri_imu_sample* s = imu_samples(h);
  const int ns = h->n;
  const double t0 = h->t0, t1 = h->t1;
  const bool fits = ns > 0 && ns <= kMaxPieces + 2 && ns <= nt;
  if (fits)
    for (int k = tid; k < ns; k += nt) W.ts[k] = s[k].t;   // one coalesced pass
  __syncthreads();
  // Zero-order-hold pieces: sample k holds on [max(t_k, t0), min(t_k+1, t1)) (the
  // last one until t1).  The pieces of positive length, in sample order, are
  // compacted by warp ballots: the same cut as a sequential walk over the interval.
  const bool cover = fits && W.ts[0] <= t0 && W.ts[ns - 1] >= t1 && t1 > t0;
  double lo = 0.0, hi = 0.0;
  bool valid = false;
  if (cover && tid < ns) {
    lo = fmax(W.ts[tid], t0);
    hi = tid + 1 < ns ? fmin(W.ts[tid + 1], t1) : t1;
    valid = hi > lo;
  }
  const unsigned ball = __ballot_sync(0xffffffffu, valid);
  if (lane == 0) W.wcount[warp] = __popc(ball);
  __syncthreads();
  if (tid == 0) {
    int tot = 0;
    for (int w = 0; w < (nt >> 5); ++w) {
      const int c = W.wcount[w];
      W.wcount[w] = tot;
      tot += c;
    }
    W.np = (cover && tot <= kMaxPieces) ? tot : -1;
  }
  __syncthreads();
  const int np = W.np;
  if (np <= 0) return false;
  if (valid) {
    const int idx = W.wcount[warp] + __popc(ball & ((1u << lane) - 1u));
    W.pk[idx] = tid;
    W.dt[idx] = hi - lo;
  }
  __syncthreads();
  // Exp(theta_k) and Jr(theta_k), one matrix element per lane (Rodrigues forms
  // I + a K + b K^2 with K = [theta]x, K^2 = theta theta^T - |theta|^2 I);
  // u_k = a_k - b_a; piece start times on the last lane
  for (int L = tid; L < 9 * np; L += nt) {
    const int k = L / 9, e = L % 9;
    const dri_imu_sample& m = s[W.pk[k]];
    const double dt = W.dt[k];
    const double th[3] = {(m.gyr[0] - bg[0]) * dt, (m.gyr[1] - bg[1]) * dt, (m.gyr[2] - bg[2]) * dt};
    const double t2 = th[0] * th[0] + th[1] * th[1] + th[2] * th[2];
    double ea, eb, jb;
    if (t2 < kSeriesT2) {
      ea = 1.0 + t2 * (-1.0 / 6 + t2 * (1.0 / 120 + t2 * (-1.0 / 5040 + t2 * (1.0 / 362880))));
      eb = 0.5 + t2 * (-1.0 / 24 + t2 * (1.0 / 720 + t2 * (-1.0 / 40320 + t2 * (1.0 / 3628800))));
      jb = 1.0 / 6 + t2 * (-1.0 / 120 + t2 * (1.0 / 5040 + t2 * (-1.0 / 362880 + t2 * (1.0 / 39916800))));
    } else {
      const double t = sqrt(t2);
      double sn, cs;
      sincos(t, &sn, &cs);
      ea = sn / t;
      eb = (1.0 - cs) / t2;
      jb = (t - sn) / (t2 * t);
    }
    const int r = e / 3, c = e % 3;
    const double K = hat_e(th, e);
    const double K2 = th[r] * th[c] - (r == c ? t2 : 0.0);
    const double id = r == c ? 1.0 : 0.0;
    W.EP[k][e] = id + ea * K + eb * K2;            // Exp
    W.Y[k][e] = id - eb * K + jb * K2;             // Jr
    if (e < 3) W.u[k][e] = m.acc[e] - ba[e];
  }
  if (tid == nt - 1) {
    double acc = 0.0;
    W.tau[0] = 0.0;
    for (int k = 0; k < np; ++k) {
      acc += W.dt[k];
      W.tau[k + 1] = acc;
    }
  }
  __syncthreads();
  // dR_{k+1} = Exp_0 ... Exp_k: inclusive prefix product (Hillis-Steele, earlier
  // factors on the left), alternating between EP and S2
  double(*cur)[9] = W.EP;
  double(*nxt)[9] = W.S2;
  for (int d = 1; d < np; d <<= 1) {
    for (int L = tid; L < 9 * np; L += nt) {
      const int k = L / 9, e = L % 9;
      nxt[k][e] = k >= d ? mm_e(cur[k - d], cur[k], e, false, false) : cur[k][e];
    }
    __syncthreads();
    double(*t)[9] = cur;
    cur = nxt;
    nxt = t;
  }
  for (int L = tid; L < 9 * (np + 1); L += nt) {
    const int k = L / 9, e = L % 9;
    W.dR[k][e] = k == 0 ? ((e % 4 == 0) ? 1.0 : 0.0) : cur[k - 1][e];
  }
  __syncthreads();
  const double T = W.tau[np];
  // Y_k <- dR_{k+1} Jr_k and u_k <- dR_k u_k (through S2 / EP), w_k
  for (int L = tid; L < 9 * np; L += nt) {
    const int k = L / 9, e = L % 9;
    W.S2[k][e] = mm_e(W.dR[k + 1], W.Y[k], e, false, false);
    if (e < 3) W.EP[k][e] = mv_e(W.dR[k], W.u[k], e, false);
    if (e == 0) W.w[k] = W.dt[k] * (T - W.tau[k + 1]) + 0.5 * W.dt[k] * W.dt[k];
  }
  __syncthreads();
  for (int L = tid; L < 9 * np; L += nt) {
    const int k = L / 9, e = L % 9;
    const double y = W.S2[k][e];
    W.Y[k][e] = y;
    if (e < 3) W.u[k][e] = W.EP[k][e];
    W.S2[k][e] = -y * W.dt[k];                     // scan input of Psi
  }
  __syncthreads();
  // Psi_k = -sum_{i<k} Y_i dt_i: inclusive additive scan, shifted by one into EP
  cur = W.S2;
  nxt = W.EP;
  for (int d = 1; d < np; d <<= 1) {
    for (int L = tid; L < 9 * np; L += nt) {
      const int k = L / 9, e = L % 9;
      nxt[k][e] = k >= d ? cur[k - d][e] + cur[k][e] : cur[k][e];
    }
    __syncthreads();
    double(*t)[9] = cur;
    cur = nxt;
    nxt = t;
  }
  if (cur == W.EP) {                                // move the result out of EP first
    for (int L = tid; L < 9 * np; L += nt) W.S2[L / 9][L % 9] = W.EP[L / 9][L % 9];
    __syncthreads();
  }
  for (int L = tid; L < 9 * (np + 1); L += nt) {
    const int k = L / 9, e = L % 9;
    W.EP[k][e] = k == 0 ? 0.0 : W.S2[k - 1][e];
  }
  if (cov && tid >= nt - 6) {                       // suffix sums for the noise transition
    const int q = tid - (nt - 6);
    const int i = q % 3;
    const bool isD = q >= 3;
    double(*Sx)[3] = isD ? W.Dv : W.Cv;
    double acc = 0.0;
    Sx[np][i] = 0.0;
    for (int k = np - 1; k >= 0; --k) {
      acc += W.u[k][i] * (isD ? W.w[k] : W.dt[k]);
      Sx[k][i] = acc;
    }
  }
  __syncthreads();
  if (warp == 0 && lane < 6) {         // dv, dp
    const int i = lane % 3;
    double acc = 0.0;
    for (int k = 0; k < np; ++k) acc += W.u[k][i] * (lane < 3 ? W.dt[k] : W.w[k]);
    (lane < 3 ? P.dv : P.dp)[i] = acc;
  } else if (warp == 1 && lane < 18) { // d(dv, dp)/d(b_g) = -sum [u_k]x Psi_k (dt_k | w_k)
    const int e = lane % 9, r = e / 3, c = e % 3, r1 = (r + 1) % 3, r2 = (r + 2) % 3;
    double acc = 0.0;
    for (int k = 0; k < np; ++k) {
      const double* u = W.u[k];
      const double* Ps = W.EP[k];
      const double hv = u[r1] * Ps[3 * r2 + c] - u[r2] * Ps[3 * r1 + c];
      acc -= hv * (lane < 9 ? W.dt[k] : W.w[k]);
    }
    (lane < 9 ? P.Vg : P.Pg)[e] = acc;
  } else if (warp == 2 && lane < 18) { // d(dv, dp)/d(b_a) = -sum dR_k (dt_k | w_k)
    const int e = lane % 9;
    double acc = 0.0;
    for (int k = 0; k < np; ++k) acc -= W.dR[k][e] * (lane < 9 ? W.dt[k] : W.w[k]);
    (lane < 9 ? P.Va : P.Pa)[e] = acc;
  } else if (warp == 3 && lane < 9) {  // d(dR)/d(b_g) = dR_N^T Psi_N
    const int r = lane / 3, c = lane % 3;
    const double* R = W.dR[np];
    const double* Ps = W.EP[np];
    P.Phig[lane] = R[r] * Ps[c] + R[3 + r] * Ps[3 + c] + R[6 + r] * Ps[6 + c];
    P.dR[lane] = R[lane];
  } else if (cov && tid >= 128 && tid < 128 + 45) {
    // covariance entry (r, c), r <= c, of (dphi, dv, dp)
    int e = tid - 128, r = 0;
    while (e >= 9 - r) { e -= 9 - r; ++r; }
    const int c = r + e;
    double acc = 0.0;
    const double q_g = gnd * gnd, q_a = and_ * and_;
    for (int k = 0; k < np; ++k) {
      const double dt = W.dt[k];
      double gr[3], gc[3];
      gyro_gain_row(W, np, k, r, gr);
      gyro_gain_row(W, np, k, c, gc);
      acc += q_g * dt * (gr[0] * gc[0] + gr[1] * gc[1] + gr[2] * gc[2]);
      if (r >= 3 && (r % 3) == (c % 3)) {   // accelerometer noise: v and p blocks
        const double ck = (T - W.tau[k + 1]) + 0.5 * dt;
        const double fr = r < 6 ? 1.0 : ck, fc = c < 6 ? 1.0 : ck;
        acc += q_a * dt * fr * fc;
      }
    }
    P.Sig[r * 9 + c] = acc;
    P.Sig[c * 9 + r] = acc;
  }
  if (tid == 0) P.T = T;
  __syncthreads();
  return true;
}

// ---------------------------------------------------------------------------
// prediction, IMU error and Jacobian
// ---------------------------------------------------------------------------

struct ImuLin {
  double R0[9], Q0[9], R1[9], Q1[9];
  double A0[9], RWS1[9], Rh[9], QA[9];
  double r[3], v[3], c[3];
  double e[18];
  double Jla[9], Jlg[9], Jra[9], Jrg[9];
  // intermediates of the lane-parallel passes
  double QR[9], Mg[9], M[9];
  double t1[3], t2[3], t3[3], t4[3], t5[3], w9[3];
  double KR[9], RP[9];
  double B[13][9];                    // Jacobian blocks, indexed by the kB* codes of imu_linearise
};

// Element e (0..8, row-major) of the rotation matrix of the unit quaternion q:
// (w^2 - |v|^2) I + 2 v v^T + 2 w [v]x.
__device__ __forceinline__ double quat_rot_e(const double* q, int e) {
  const int r = e / 3, c = e % 3;
  const double w = q[0];
  double m = 2.0 * q[1 + r] * q[1 + c];
  if (r == c) m += w * w - (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  else m += 2.0 * w * ((((c - r + 3) % 3) == 1) ? -q[4 - r - c] : q[4 - r - c]);
  return m;
}

// component i of the rotation vector of R (so3_log, as one lane's share)
__device__ __forceinline__ double log_i(const double* R, int i) {
  const double c = 0.5 * (R[0] + R[4] + R[8] - 1.0);
  const double v0 = R[7] - R[5], v1 = R[2] - R[6], v2 = R[3] - R[1];
  double f;
  if (c > 0.99875) {
    const double s2 = 0.25 * (v0 * v0 + v1 * v1 + v2 * v2);
    f = 0.5 * (1.0 + s2 * (1.0 / 6 + s2 * (3.0 / 40 + s2 * (5.0 / 112 + s2 * (35.0 / 1152 +
               s2 * (63.0 / 2816 + s2 * (231.0 / 13312)))))));
  } else {
    const double t = acos(fmin(1.0, fmax(-1.0, c)));
    f = t / (2.0 * sin(t));
  }
  return f * (i == 0 ? v0 : i == 1 ? v1 : v2);
}
// element e of Jl^-1(s w) (s = +1, or -1 for Jr^-1(w) = Jl^-1(-w))
__device__ __forceinline__ double jlinv_e(const double* w0, double s, int e) {
  const double w[3] = {s * w0[0], s * w0[1], s * w0[2]};
  const double t2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double c;
  if (t2 < kSeriesT2) {
    c = 1.0 / 12 + t2 * (1.0 / 720 + t2 * (1.0 / 30240 + t2 * (1.0 / 1209600 + t2 * (1.0 / 47900160))));
  } else {
    const double t = sqrt(t2);
    double sn, co;
    sincos(t, &sn, &co);
    c = 1.0 / t2 - (1.0 + co) / (2.0 * t * sn);
  }
  const int r = e / 3, q = e % 3;
  // I - K/2 + c K^2,  K^2 = w w^T - t2 I
  return (r == q ? 1.0 - c * t2 : 0.0) - 0.5 * hat_e(w, e) + c * w[r] * w[q];
}

// Jacobian-block codes of imu_linearise: 0 zero, 1 +I, 2 -I, 16 + 2 m + neg: block B[m] / J*
constexpr int kBJra = 0, kBJrg = 1, kB7 = 2, kBJla = 3, kB9 = 4, kB10 = 5, kB12 = 6, kB13 = 7,
              kB14 = 8, kB16 = 9, kB17 = 10, kB19 = 11, kB20 = 12, kBJlg = 13;
__device__ constexpr unsigned char kJBlk[2][6][6] = {
    // x0 columns: r, alpha, v, b_g, b_a, gravity (2 columns)
    {{1, 16 + 2 * kB7, 16 + 2 * kB10, 16 + 2 * kB12, 16 + 2 * kB16, 16 + 2 * kB19},
     {0, 16 + 2 * kBJla, 0, 16 + 2 * kB13, 0, 0},
     {0, 16 + 2 * kB9, 1, 16 + 2 * kB14, 16 + 2 * kB17, 16 + 2 * kB20},
     {0, 0, 0, 1, 0, 0},
     {0, 0, 0, 0, 1, 0},
     {0, 0, 0, 0, 0, 16 + 2 * kBJlg}},
    // x1 columns
    {{2, 0, 0, 0, 0, 0},
     {0, 17 + 2 * kBJra, 0, 0, 0, 0},
     {0, 0, 2, 0, 0, 0},
     {0, 0, 0, 2, 0, 0},
     {0, 0, 0, 0, 2, 0},
     {0, 0, 0, 0, 0, 17 + 2 * kBJrg}}};

// Whole block: prediction x^1(x0), error e = x^1 boxminus x1 and (when J) the
// 18 x 2 ns Jacobian (row-major; columns: x0 tangent 0..ns-1, x1 tangent
// ns..2 ns-1; ns = 17 keeps the x and y columns of the gravity blocks, 18 all
// three).
// Warp 0 runs the chain of small products one output element per lane, up to
// three independent products per pass (lanes 0-8, 9-17, 18-26).
//   R^ = R0 Rc dR Rc^T,  r^ = r0 + R0 rc + Q0^T c + A0 dp - R^ rc  (A0 = R0 Rc),
//   v^ = v0 + g T + Q0 A0 dv,  c = v0 T + g T^2 / 2,
//   e = (r^ - r1, log(R^ R1^T), v^ - v1, b0 - b1, log(Q0 Q1^T)).
__device__ void imu_linearise(const DState& x0, const DState& x1, const Preint& P,
                              const SolveParams& sp, ImuLin& L, double* J, int ns = 17) {
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int g3 = lane / 9, e9 = lane % 9;
  const double T = P.T;
  const double* Rc = sp.R_CS;
  const double* rc = sp.r_CS;
  if (warp == 0) {
    // rotations of the four quaternions, c
    if (lane < 27) (g3 == 0 ? L.R0 : g3 == 1 ? L.Q0 : L.R1)[e9] =
        quat_rot_e(g3 == 0 ? x0.q : g3 == 1 ? x0.qg : x1.q, e9);
    __syncwarp();
    if (lane < 9) L.Q1[lane] = quat_rot_e(x1.qg, lane);
    else if (lane < 12) L.c[lane - 9] = x0.v[lane - 9] * T + (lane == 11 ? -0.5 * sp.g * T * T : 0.0);
    else if (lane < 18) L.e[9 + lane - 12] = lane < 15 ? x0.bg[lane - 12] - x1.bg[lane - 12]
                                                       : x0.ba[lane - 15] - x1.ba[lane - 15];
    __syncwarp();
    // A0 = R0 Rc, QR = Q0 R0, Mg = Q0 Q1^T
    if (lane < 27) {
      const double* A = g3 == 0 ? L.R0 : L.Q0;
      const double* B = g3 == 0 ? Rc : g3 == 1 ? L.R0 : L.Q1;
      (g3 == 0 ? L.A0 : g3 == 1 ? L.QR : L.Mg)[e9] = mm_e(A, B, e9, false, g3 == 2);
    }
    __syncwarp();
    // RWS1 = A0 dR, QA = QR Rc, t1 = R0 rc, t2 = Q0^T c, t3 = A0 dp
    if (lane < 18) {
      (g3 == 0 ? L.RWS1 : L.QA)[e9] = mm_e(g3 == 0 ? L.A0 : L.QR, g3 == 0 ? P.dR : Rc, e9, false, false);
    } else if (lane < 27) {
      const int k = (lane - 18) / 3, i = (lane - 18) % 3;
      const double* A = k == 0 ? L.R0 : k == 1 ? L.Q0 : L.A0;
      const double* x = k == 0 ? rc : k == 1 ? L.c : P.dp;
      (k == 0 ? L.t1 : k == 1 ? L.t2 : L.t3)[i] = mv_e(A, x, i, k == 1);
    }
    __syncwarp();
    // Rh = RWS1 Rc^T, t5 = QA dv, w9 = A0 dv
    if (lane < 9) L.Rh[lane] = mm_e(L.RWS1, Rc, lane, false, true);
    else if (lane < 15) {
      const int k = (lane - 9) / 3, i = (lane - 9) % 3;
      (k == 0 ? L.t5 : L.w9)[i] = mv_e(k == 0 ? L.QA : L.A0, P.dv, i, false);
    }
    __syncwarp();
    // t4 = Rh rc, M = Rh R1^T, v^, e_v
    if (lane < 3) L.t4[lane] = mv_e(L.Rh, rc, lane, false);
    else if (lane < 12) L.M[lane - 3] = mm_e(L.Rh, L.R1, lane - 3, false, true);
    else if (lane < 15) {
      const int i = lane - 12;
      const double vi = x0.v[i] + (i == 2 ? -sp.g : 0.0) * T + L.t5[i];
      L.v[i] = vi;
      L.e[6 + i] = vi - x1.v[i];
    }
    __syncwarp();
    // r^, e_r; e_a = log(R^ R1^T), e_g = log(Q0 Q1^T)
    if (lane < 3) {
      const double ri = x0.r[lane] + L.t1[lane] + L.t2[lane] + L.t3[lane] - L.t4[lane];
      L.r[lane] = ri;
      L.e[lane] = ri - x1.r[lane];
    } else if (lane < 9) {
      const int k = (lane - 3) / 3, i = (lane - 3) % 3;
      L.e[(k == 0 ? 3 : 15) + i] = log_i(k == 0 ? L.M : L.Mg, i);
    }
    __syncwarp();
  }
  __syncthreads();
  if (J == nullptr) return;
  // Jacobians of the two orientation errors, and the product blocks (warps 0-1)
  if (warp == 0) {
    if (lane < 27) (g3 == 0 ? L.Jla : g3 == 1 ? L.Jlg : L.Jra)[e9] =
        jlinv_e(g3 == 1 ? L.e + 15 : L.e + 3, g3 == 2 ? -1.0 : 1.0, e9);
    __syncwarp();
    if (lane < 9) L.Jrg[lane] = jlinv_e(L.e + 15, -1.0, lane);
    __syncwarp();
    // B13 = Jla RWS1 Phig (via RP), B14 = QA Vg, B16 = A0 Pa
    if (lane < 9) L.RP[lane] = mm_e(L.RWS1, P.Phig, lane, false, false);
    else if (lane < 18) L.B[kB14][e9] = mm_e(L.QA, P.Vg, e9, false, false);
    else if (lane < 27) L.B[kB16][e9] = mm_e(L.A0, P.Pa, e9, false, false);
    __syncwarp();
    if (lane < 9) L.B[kB13][lane] = mm_e(L.Jla, L.RP, lane, false, false);
    __syncwarp();
  } else if (warp == 1) {
    // B12 = A0 Pg + [Rh rc]x RWS1 Phig (via KR), B17 = QA Va
    if (lane < 9) L.KR[lane] = hatm_e(L.t4, L.RWS1, lane);
    else if (lane < 18) L.B[kB17][e9] = mm_e(L.QA, P.Va, e9, false, false);
    __syncwarp();
    if (lane < 9) L.B[kB12][lane] = mm_e(L.A0, P.Pg, lane, false, false) + mm_e(L.KR, P.Phig, lane, false, false);
    __syncwarp();
  } else if (warp == 2) {
    // B7 = -[r^ - r0 - Q0^T c]x, B9 = -Q0 [A0 dv]x, B10 = T Q0^T
    if (lane < 9) {
      const double u[3] = {L.r[0] - x0.r[0] - L.t2[0], L.r[1] - x0.r[1] - L.t2[1], L.r[2] - x0.r[2] - L.t2[2]};
      L.B[kB7][lane] = -hat_e(u, lane);
    } else if (lane < 18) {
      L.B[kB9][e9] = -mhat_e(L.Q0, false, L.w9, e9);
    } else if (lane < 27) {
      L.B[kB10][e9] = T * L.Q0[3 * (e9 % 3) + e9 / 3];
    }
    __syncwarp();
  } else if (warp == 3) {
    // B19 = Q0^T [c]x, B20 = -[Q0 A0 dv]x (first two columns used)
    if (lane < 9) L.B[kB19][lane] = mhat_e(L.Q0, true, L.c, lane);
    else if (lane < 18) L.B[kB20][e9] = -hat_e(L.t5, e9);
    __syncwarp();
  }
  __syncthreads();
  const double* src[14] = {L.Jra, L.Jrg, L.B[kB7], L.Jla, L.B[kB9], L.B[kB10], L.B[kB12],
                           L.B[kB13], L.B[kB14], L.B[kB16], L.B[kB17], L.B[kB19], L.B[kB20], L.Jlg};
  const int nj = 2 * ns;
  for (int idx = tid; idx < 18 * nj; idx += blockDim.x) {
    const int r = idx / nj, col = idx % nj;
    const int side = col >= ns ? 1 : 0, cl = col - ns * side;
    const int cg = cl < 15 ? cl / 3 : 5, cc = cl < 15 ? cl % 3 : cl - 15;
    const int rb = r / 3, rr = r % 3;
    const int code = kJBlk[side][rb][cg];
    double v = 0.0;
    if (code == 1 || code == 2) v = rr == cc ? (code == 1 ? 1.0 : -1.0) : 0.0;
    else if (code >= 16) {
      const double m = src[(code - 16) >> 1][3 * rr + cc];
      v = (code & 1) ? -m : m;
    }
    J[idx] = v;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// state algebra
// ---------------------------------------------------------------------------

__device__ void load_pose_ref(Ctrl* c) {
  quat_to_rot(c->x.q, c->Rref);
  for (int i = 0; i < 3; ++i) c->rref[i] = c->x.r[i];
}

// ---------------------------------------------------------------------------
// warp-cooperative state algebra
// ---------------------------------------------------------------------------
// An FP64 warp instruction costs the same whatever its active lanes, so the
// small vector / quaternion / 3x3 algebra of the states runs one element per
// lane: a quaternion product is 4 FMAs on 4 lanes instead of 16 on one.

// Component k (0..3) of the Hamilton product a (x) b: the b index of a_j is
// k ^ j, and the sign pattern of the sixteen terms is the bit mask 0x428E.
__device__ __forceinline__ double quat_mul_k(const double a[4], const double* b, int k,
                                             bool conj_b) {
  double o = 0.0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int m = k ^ j;
    const double bm = (conj_b && m) ? -b[m] : b[m];
    const double t = ((0x428E >> (4 * k + j)) & 1) ? -a[j] : a[j];
    o = fma(t, bm, o);
  }
  return o;
}


// 2 asin(s) / s for s^2 below 6.25e-4 (s = sin(theta / 2), theta < 0.05): the
// angle / |v| factor of a unit quaternion's log, from the series of asin.
__device__ __forceinline__ double quat_log_factor(double s2, double w) {
  if (s2 < 6.25e-4)
    return 2.0 * (1.0 + s2 * (1.0 / 6 + s2 * (3.0 / 40 + s2 * (5.0 / 112 + s2 * (35.0 / 1152 +
                                                                                 s2 * (63.0 / 2816))))));
  const double s = sqrt(s2);
  return 2.0 * atan2(s, w) / s;
}

// x <- x boxplus d (Eq. 2) by one warp; x, d in shared or global memory.  Lanes
// 0-11 add the vector parts; lanes 0-3 update q with d[3..5], lanes 4-7 q_IW
// with (d[15], d[16], 0), or d[15..17] with g3 (3-D gravity): q <- exp(d) (x) q,
// renormalised.
__device__ void warp_state_boxplus(DState& x, const double* d, bool g3 = false) {
  const int lane = threadIdx.x & 31;
  const int grp = (lane >> 2) & 1, k = lane & 3;
  double* q = grp ? x.qg : x.q;
  const double d0 = grp ? d[15] : d[3], d1 = grp ? d[16] : d[4], d2 = grp ? (g3 ? d[17] : 0.0) : d[5];
  const double t2 = d0 * d0 + d1 * d1 + d2 * d2;
  double sh, ch;
  if (t2 < kSeriesT2) {
    sh = 0.5 + t2 * (-1.0 / 48 + t2 * (1.0 / 3840 + t2 * (-1.0 / 645120 + t2 * (1.0 / 185794560))));
    ch = 1.0 + t2 * (-1.0 / 8 + t2 * (1.0 / 384 + t2 * (-1.0 / 46080 + t2 * (1.0 / 10321920))));
  } else {
    const double t = sqrt(t2);
    double sn, cs;
    sincos(0.5 * t, &sn, &cs);
    sh = sn / t;
    ch = cs;
  }
  const double e[4] = {ch, sh * d0, sh * d1, sh * d2};
  double o = quat_mul_k(e, q, k, false);
  double n2 = o * o;
  n2 += __shfl_xor_sync(0xffffffffu, n2, 1);
  n2 += __shfl_xor_sync(0xffffffffu, n2, 2);
  o *= fabs(n2 - 1.0) < 1e-6 ? 1.5 - 0.5 * n2 : rsqrt(n2);
  __syncwarp();
  if (lane < 8) q[k] = o;
  if (lane < 12) {
    const int g = lane / 3, i = lane % 3;
    double* v = g == 0 ? x.r : g == 1 ? x.v : g == 2 ? x.bg : x.ba;
    v[i] += d[(g == 0 ? 0 : 3 + 3 * g) + i];
  }
  __syncwarp();
}

// d = x boxminus y (17, or 18 with g3) by one warp: vector parts subtract; orientations
// log(q_x (x) q_y^-1) (lanes 0-3), gravity the x, y (with g3 also z) of log(qg_x (x) qg_y^-1)
// (lanes 4-7) -- the rotation vector of R_x R_y^T, taken with w >= 0.
__device__ void warp_state_boxminus(const DState& x, const DState& y, double* d, bool g3 = false) {
  const int lane = threadIdx.x & 31;
  const int grp = (lane >> 2) & 1, k = lane & 3;
  const double* qx = grp ? x.qg : x.q;
  const double* qy = grp ? y.qg : y.q;
  const double a[4] = {qx[0], qx[1], qx[2], qx[3]};
  double o = quat_mul_k(a, qy, k, true);
  const int base = lane & ~3;
  const double w = __shfl_sync(0xffffffffu, o, base);
  if (w < 0.0) o = -o;
  double s2 = k ? o * o : 0.0;
  s2 += __shfl_xor_sync(0xffffffffu, s2, 1);
  s2 += __shfl_xor_sync(0xffffffffu, s2, 2);
  const double f = quat_log_factor(s2, fabs(w));
  if (lane < 12) {
    const int g = lane / 3, i = lane % 3;
    const double* vx = g == 0 ? x.r : g == 1 ? x.v : g == 2 ? x.bg : x.ba;
    const double* vy = g == 0 ? y.r : g == 1 ? y.v : g == 2 ? y.bg : y.ba;
    d[(g == 0 ? 0 : 3 + 3 * g) + i] = vx[i] - vy[i];
  }
  if (grp == 0 && k > 0 && lane < 4) d[2 + k] = f * o;
  if (grp == 1 && k > 0 && (k < 3 || g3) && lane < 8) d[14 + k] = f * o;
  __syncwarp();
}

// Pixel-kernel transforms for the next linearisation (FP64 -> FP32), one warp:
// A = R_ref^T R_1 - I, t = R_ref^T (r_1 - r_ref) and A_0 = R_0^T R_1 - I,
// t_0 = R_0^T (r_1 - r_0).  R_0, R_1 go through shared scratch rot[18].
__device__ void warp_write_transforms(Ctrl* c, const DState& x0, const DState& x1, double* rot) {
  const int lane = threadIdx.x & 31;
  if (lane < 18) rot[lane] = quat_rot_e(lane < 9 ? x1.q : x0.q, lane % 9);
  __syncwarp();
  const double* R1 = rot;
  const double* R0 = rot + 9;
  if (lane < 18) {
    const int e = lane % 9, r = e / 3, cc = e % 3;
    const double* M = lane < 9 ? c->Rref : R0;
    double v = (r == cc) ? -1.0 : 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) v = fma(M[3 * k + r], R1[3 * k + cc], v);
    (lane < 9 ? c->xf_icp : c->xf_rgb)[e] = (float)v;
  } else if (lane < 24) {
    const int i = (lane - 18) % 3;
    const bool icp = lane < 21;
    const double* M = icp ? c->Rref : R0;
    const double* o = icp ? c->rref : x0.r;
    double v = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) v = fma(M[3 * k + i], x1.r[k] - o[k], v);
    (icp ? c->xf_icp : c->xf_rgb)[9 + i] = (float)v;
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// dense symmetric factorisation
// ---------------------------------------------------------------------------

// In-place LDL^T of the symmetric n x n matrix in A (lower triangle read): the
// strict lower triangle becomes the unit-lower L, the diagonal D.  Whole block;
// col is shared scratch of 2 n doubles, fail a shared int.  False (for all
// threads) if a pivot is not positive.
__device__ bool block_ldlt(double* A, int n, int ld, double* col, int* fail) {
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) *fail = 0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    const double d = A[k * ld + k];
    if (tid == 0 && !(d > 0.0 && d < INFINITY)) *fail = 1;
    double* ck = col + (k & 1) * n;
    const double* cp = col + ((k + 1) & 1) * n;
    for (int i = k + 1 + tid; i < n; i += nt) ck[i] = A[i * ld + k] / d;
    if (k > 0)
      for (int i = k + tid; i < n; i += nt) A[i * ld + (k - 1)] = cp[i];
    __syncthreads();
    const int m = n - k - 1;
    for (int p = tid; p < m * m; p += nt) {
      const int i = k + 1 + p / m, j = k + 1 + p % m;
      if (j <= i) A[i * ld + j] -= A[i * ld + k] * ck[j];
    }
    __syncthreads();
  }
  return *fail == 0;
}

// The same for one right-hand side in one thread.
__device__ void ldlt_solve_thread(const double* A, int n, int ld, double* b) {
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= A[i * ld + k] * b[k];
    b[i] = s;
  }
  for (int i = 0; i < n; ++i) b[i] /= A[i * ld + i];
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int k = i + 1; k < n; ++k) s -= A[k * ld + i] * b[k];
    b[i] = s;
  }
}

// Pivot reciprocal: an FP32 seed refined by one Newton-Raphson step (relative
// error below 2^-45; the factorisation is then exact for a matrix whose pivots
// are perturbed by that amount, far below what the system's rounding already
// costs).  The seed's conversions are integer operations on the bit patterns
// (the leading 23 mantissa bits of d, the exponent re-biased between the
// formats; d and 1 / d are normal in both here): on this GPU every FP64-pipe
// instruction on the pivot's dependency chain costs tens of cycles.
__device__ __forceinline__ double pivot_recip(double d) {
  if (d > 1e-30 && d < 1e30) {
    const int hi = __double2hiint(d);
    const unsigned lo = (unsigned)__double2loint(d);
    const float f = __int_as_float((int)(((unsigned)hi - 0x38000000u) << 3 | lo >> 29));
    const int yb = __float_as_int(__frcp_rn(f));
    const double y = __hiloint2double((yb >> 3) + 0x38000000, (int)((unsigned)yb << 29));
    return fma(y, fma(-d, y, 1.0), y);
  }
  return 1.0 / d;
}

// Solves A x = b for a symmetric positive definite N x N matrix (row-major in
// shared memory, lower triangle read) on the first T threads (T a multiple of 32;
// the other threads of the block must not call it).  Element-parallel LDL^T: every
// thread keeps its share of the lower triangle of [A | b] in registers; per pivot
// the column is published in a double-buffered shared vector behind one named
// barrier, and every warp computes the pivot reciprocal itself (no second
// barrier).  The forward substitution is the b column of the same sweep; the
// backward substitution runs in warp 0 with shuffles.  On this GPU an FP64 warp
// instruction occupies its SM sub-partition's FP64 unit for ~64 cycles whatever
// the number of active lanes, so the work is spread over the lanes of T/32 warps
// on different sub-partitions.  Scratch: colbuf 2 (N + 1), Lsm N * N, piv N.
// Returns false (in every calling thread) if a pivot is not positive.
//
// NS > 0 splits the sweep for a system whose trailing (N - NS) x (N - NS) block
// and right-hand side still lack an additive term that is not known yet: the
// first NS pivots run on what A and b hold, which leaves the Schur complement
// of the leading block in the trailing entries; then the calling threads wait
// for the preceding kernel (grid dependency) and for the other T threads of the
// block (barrier 2 over 2 T threads), which publish the missing term in Padd
// ((N - NS) x (N - NS), full) and gadd (N - NS); the owners add it to their
// trailing entries and the sweep finishes.  Elimination order does not matter
// for an additive update of entries that no earlier pivot reads.
template <int N, int T, int NS = 0>
__device__ bool ep_ldlt_solve(const double* A, const double* b, double* x, double* colbuf,
                              double* Lsm, double* piv, const double* Padd = nullptr,
                              const double* gadd = nullptr) {
  constexpr int kEnt = N * (N + 1) / 2 + N;          // lower triangle + the b column
  constexpr int kOwn = (kEnt + T - 1) / T;
  const int t = threadIdx.x;
  int ei[kOwn], ej[kOwn];
  double v[kOwn];
#pragma unroll
  for (int o = 0; o < kOwn; ++o) {
    const int e = t + o * T;
    int i = -1, j = -1;
    if (e < kEnt) {
      // entries dealt out by lifetime: group g (column c = N - 1 - g) holds
      // (c..N-1, c) and the right-hand side's (c, N), g + 2 entries, updated
      // by pivots 0..c-1; groups in order of decreasing c, so the entries a
      // pivot still updates are a prefix of the threads and fill the fewest
      // warps (an FP64 warp instruction costs the same with 1 or 32 lanes)
      int g = (int)((sqrtf(9.0f + 8.0f * e) - 3.0f) * 0.5f);
      while (g * (g + 3) / 2 > e) --g;
      while ((g + 1) * (g + 4) / 2 <= e) ++g;
      const int r = e - g * (g + 3) / 2, c = N - 1 - g;
      i = r <= g ? c + r : c;
      j = r <= g ? c : N;
    }
    ei[o] = i;
    ej[o] = j;
    v[o] = (i < 0) ? 0.0 : (j == N ? b[i] : A[i * N + j]);
  }
  for (int k = 0; k < N; ++k) {
    if (NS > 0 && k == NS) {
      grid_dep_wait();
      asm volatile("bar.sync 2, %0;" ::"n"(2 * T) : "memory");
#pragma unroll
      for (int o = 0; o < kOwn; ++o) {
        const int i = ei[o], j = ej[o];
        if (i >= NS && j >= NS) v[o] += j == N ? gadd[i - NS] : Padd[(i - NS) * (N - NS) + (j - NS)];
      }
    }
    double* cb = colbuf + (k & 1) * (N + 1);
#pragma unroll
    for (int o = 0; o < kOwn; ++o) {
      if (ej[o] == k) cb[ei[o]] = v[o];              // column k (unscaled) with the pivot
      if (ej[o] == N && ei[o] == k) cb[N] = v[o];    // z_k
    }
    asm volatile("bar.sync 1, %0;" ::"n"(T) : "memory");
    const double d = cb[k];
    const double r = pivot_recip(d);
    const double zk = cb[N];
    if (t == 0) {
      piv[k] = d;
      x[k] = zk * r;                                 // y_k = z_k / d_k
    }
#pragma unroll
    for (int o = 0; o < kOwn; ++o) {
      const int i = ei[o], j = ej[o];
      if (i > k && j > k) v[o] = fma(-(cb[i] * r), j == N ? zk : cb[j], v[o]);
    }
  }
  // unit-lower L = column k divided by d_k (v still holds the unscaled columns)
#pragma unroll
  for (int o = 0; o < kOwn; ++o) {
    const int i = ei[o], j = ej[o];
    if (i >= 0 && j < i) Lsm[i * N + j] = v[o] * pivot_recip(piv[j]);
  }
  asm volatile("bar.sync 1, %0;" ::"n"(T) : "memory");
  bool ok = true;
  if (t < 32) {                                      // L^T x = y
    const int lane = t;
    double y0 = (lane < N) ? x[lane] : 0.0;
    double y1 = (lane + 32 < N) ? x[lane + 32] : 0.0;
    for (int k = N - 1; k > 0; --k) {
      const double xk = __shfl_sync(0xffffffffu, k < 32 ? y0 : y1, k & 31);
      if (lane < k) y0 = fma(-Lsm[k * N + lane], xk, y0);
      if (lane + 32 < k) y1 = fma(-Lsm[k * N + lane + 32], xk, y1);
    }
    if (lane < N) x[lane] = y0;
    if (lane + 32 < N) x[lane + 32] = y1;
    bool good = true;
    for (int k = lane; k < N; k += 32) good = good && piv[k] > 0.0 && piv[k] < INFINITY;
    ok = __all_sync(0xffffffffu, good);
  }
  asm volatile("bar.sync 1, %0;" ::"n"(T) : "memory");
  if (t < 32 && t == 0) colbuf[0] = ok ? 1.0 : 0.0;
  asm volatile("bar.sync 1, %0;" ::"n"(T) : "memory");
  return colbuf[0] != 0.0;
}

// ---------------------------------------------------------------------------
// joint system (Eq. 6-7)
// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------
// First-order bias update of the pre-integration (DRI_IMU_FIRST_ORDER)
// ---------------------------------------------------------------------------

// Stores a pre-integration and its biases as the frame's linearisation point.
__device__ void store_lin(Ctrl* c, const Preint& P, const double* bg, const double* ba) {
  const int tid = threadIdx.x;
  const double* src[8] = {P.dR, P.dv, P.dp, P.Phig, P.Vg, P.Pg, P.Va, P.Pa};
  const int off[9] = {0, 9, 12, 15, 24, 33, 42, 51, 60};
  if (tid < 60) {
    int k = 0;
    while (tid >= off[k + 1]) ++k;
    c->pre_lin[tid] = src[k][tid - off[k]];
  } else if (tid == 60) {
    c->pre_lin[60] = P.T;
  } else if (tid >= 64 && tid < 70) {
    c->b_lin[tid - 64] = tid < 67 ? bg[tid - 64] : ba[tid - 67];
  }
}

// The pre-integration of this iteration at x0's biases (bg, ba) from the
// linearisation point (Forster et al.'s first-order update):
//   dR = dR_lin Exp(Phi_g dbg),  dv = dv_lin + V_g dbg + V_a dba,
//   dp = dp_lin + P_g dbg + P_a dba,  Phi_g <- Jr(Phi_g dbg) Phi_g
// (the rotation's bias Jacobian at the updated point; the others are linear).
// Once |dbg| > relin_g or |dba| > relin_a the samples are re-integrated at
// (bg, ba), which become the linearisation point.  Whole block; P in shared
// memory; `scratch` 19 doubles of shared memory.
__device__ bool preint_first_order(const SolveParams& sp, Ctrl* c, const double* bg,
                                   const double* ba, ImuWork& W, Preint& P, double* scratch) {
  const int tid = threadIdx.x;
  double dbg[3], dba[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    dbg[i] = bg[i] - c->b_lin[i];
    dba[i] = ba[i] - c->b_lin[3 + i];
  }
  const double ng = sqrt(dbg[0] * dbg[0] + dbg[1] * dbg[1] + dbg[2] * dbg[2]);
  const double na = sqrt(dba[0] * dba[0] + dba[1] * dba[1] + dba[2] * dba[2]);
  if (ng > sp.relin_g || na > sp.relin_a) {      // uniform over the block
    const bool ok = preintegrate_block(sp.imu, bg, ba, false, 0.0, 0.0, W, P);
    if (ok) store_lin(c, P, bg, ba);
    return ok;
  }
  const double* L = c->pre_lin;
  double* th = scratch;                          // Phi_g dbg (3), Exp (9), Jr (9)... in place
  double* E = scratch + 3;
  double* Jrm = scratch + 12;
  // lanes 0-2: theta; 3-8: dv, dp; 9-44: V_g, P_g, V_a, P_a copied; 45: T
  if (tid < 3) {
    th[tid] = L[15 + 3 * tid] * dbg[0] + L[16 + 3 * tid] * dbg[1] + L[17 + 3 * tid] * dbg[2];
  } else if (tid < 9) {
    const int q = tid - 3, i = q % 3;
    const double* M = q < 3 ? L + 24 : L + 33;   // V_g or P_g
    const double* N = q < 3 ? L + 42 : L + 51;   // V_a or P_a
    double v = L[(q < 3 ? 9 : 12) + i];
#pragma unroll
    for (int j = 0; j < 3; ++j) v = fma(M[3 * i + j], dbg[j], fma(N[3 * i + j], dba[j], v));
    (q < 3 ? P.dv : P.dp)[i] = v;
  } else if (tid < 45) {
    const int q = tid - 9, m = q / 9, e = q % 9;
    (m == 0 ? P.Vg : m == 1 ? P.Pg : m == 2 ? P.Va : P.Pa)[e] = L[24 + q];
  } else if (tid == 45) {
    P.T = L[60];
  }
  __syncthreads();
  if (tid < 9) {                                 // Exp(theta), Jr(theta): one element per lane
    const double t2 = th[0] * th[0] + th[1] * th[1] + th[2] * th[2];
    double ea, eb, jb;
    if (t2 < kSeriesT2) {
      ea = 1.0 + t2 * (-1.0 / 6 + t2 * (1.0 / 120 + t2 * (-1.0 / 5040 + t2 * (1.0 / 362880))));
      eb = 0.5 + t2 * (-1.0 / 24 + t2 * (1.0 / 720 + t2 * (-1.0 / 40320 + t2 * (1.0 / 3628800))));
      jb = 1.0 / 6 + t2 * (-1.0 / 120 + t2 * (1.0 / 5040 + t2 * (-1.0 / 362880 + t2 * (1.0 / 39916800))));
    } else {
      const double t = sqrt(t2);
      double sn, cs;
      sincos(t, &sn, &cs);
      ea = sn / t;
      eb = (1.0 - cs) / t2;
      jb = (t - sn) / (t2 * t);
    }
    const int r = tid / 3, q = tid % 3;
    const double K = hat_e(th, tid);
    const double K2 = th[r] * th[q] - (r == q ? t2 : 0.0);
    const double id = r == q ? 1.0 : 0.0;
    E[tid] = id + ea * K + eb * K2;
    Jrm[tid] = id - eb * K + jb * K2;
  }
  __syncthreads();
  if (tid < 9) {
    P.dR[tid] = mm_e(L, E, tid, false, false);
  } else if (tid >= 32 && tid < 41) {
    P.Phig[tid - 32] = mm_e(Jrm, L + 15, tid - 32, false, false);
  }
  __syncthreads();
  return true;
}

struct GnSmem {
  ImuWork W;
  Preint P;
  ImuLin L;
  DState x0, x1;
  double J[18 * 34];
  double WJa[9 * 26];                 // W_9 J rows 0..8, columns 0..25 (the non-zero ones)
  double We[9];
  double H[34 * 34];
  double A[34 * 34];
  double b[34], x[34], scale[34];
  double Hl[2][36];                   // world-frame 6x6 of ICP, photometric (weighted)
  double gl[2][6];
  double M6[36], MH6[36];
  double P12[144], g12[12];           // the pixel terms on the poses of (x0, x1), full
  double dprior[17];
  double Hr[26 * 26], br[26];          // reduced system (x1's bias / gravity eliminated)
  double xr[26], piv[26];
  double col[2 * 27];
  double Lsm[26 * 26];                // L rows of the solver
  double fo[21];                      // first-order bias update scratch
  double Bg[6], Ag[6];                // gravity Jacobian blocks of x1 and x0 (3 x 2)
  double rot[18];                     // R_1, R_0 of the pixel transforms
  double cost_imu;
  int ok, fail, pd;
};

// Gyro-only variant (DRI_TRACK_GYRO_ONLY): tangent component k (0..33) of the
// joint state is held -- velocity (6..8), accelerometer bias (12..14) and
// gravity (15, 16) of either state, which nothing measures without the
// accelerometer rows.
__device__ __forceinline__ bool held_gyro_only(int k) {
  const int m = k < 17 ? k : k - 17;
  return (m >= 6 && m < 9) || m >= 12;
}

// Margin decisions the pixel kernel counted (its launch for a level's last
// iteration counts them; the others add nothing): stored for the level, and
// the accumulator cleared for the next launch.
__device__ __forceinline__ void store_margin(Ctrl* c, int level) {
  c->n_margin[level] = (int32_t)(c->margin_acc[0] + c->margin_acc[1]);
  c->margin_acc[0] = c->margin_acc[1] = 0u;
}

// Assemble the joint system at (ctrl->x0, ctrl->x1) into S.H (full), S.b.
// Entry e (0..71) of the two pixel systems rotated into W: term e / 36 (0 ICP
// with R_ref, 1 photometric with R_0), element e % 36 of its 6x6 (and, for
// column 0, the row of its 6-vector), weighted by W_ICP / W_RGB.
template <class Smem>
__device__ void pixel_system_entry(const SolveParams& sp, const Ctrl* c, Smem& S, int e) {
  const int term = e / 36, idx = e % 36;
  const int i = idx / 6, j = idx % 6;
  double R[9];
  if (term == 0) {
    for (int k = 0; k < 9; ++k) R[k] = c->Rref[k];
  } else {
    quat_to_rot(c->x0.q, R);
  }
  const double* s = c->sums + term * kSums;
  auto hloc = [&](int a, int b) {
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    return s[lo * 6 - lo * (lo - 1) / 2 + (hi - lo)];
  };
  // Hw = Q Hloc Q^T with Q = diag(R, R)
  double acc = 0.0;
  const int bi = i / 3, ri = i % 3, bj = j / 3, rj = j % 3;
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l) acc += R[ri * 3 + k] * hloc(bi * 3 + k, bj * 3 + l) * R[rj * 3 + l];
  const double w = term == 0 ? sp.W_icp : sp.W_rgb;
  S.Hl[term][idx] = w * acc;
  if (j == 0) {
    double g = 0.0;
    for (int k = 0; k < 3; ++k) g += R[ri * 3 + k] * s[21 + bi * 3 + k];
    S.gl[term][i] = -w * g;
  }
}


// State-only part of the joint system (Eq. 7 without the pixel terms) at
// (ctrl->x0, ctrl->x1): the IMU term (Eq. 5-6), the prior on x0, and the
// reduced system with x1's biases and gravity eliminated in closed form.
// Whole block.  Reads no pixel sum, so it runs while the preceding pixel kernel
// is still at work.  Leaves the upper triangle of the full 34-dimensional S.H,
// S.b, the reduced 26-dimensional S.Hr (full), S.br, and S.cost_imu; S.ok false
// (in every thread) if the IMU samples do not cover the interval.
__device__ void assemble_state(const SolveParams& sp, GnSmem& S) {
  Ctrl* c = sp.ctrl;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) {
    S.x0 = c->x0;
    S.x1 = c->x1;
  }
  if ((tid >> 5) == 4) {
    warp_state_boxminus(c->x0, c->xbar, S.dprior);
  } else if (tid == 160) {
    for (int i = 0; i < 36; ++i) S.M6[i] = (i % 7 == 0) ? 1.0 : 0.0;
    const double d[3] = {c->x1.r[0] - c->x0.r[0], c->x1.r[1] - c->x0.r[1], c->x1.r[2] - c->x0.r[2]};
    double K[9];
    hat3(d, K);
    for (int r = 0; r < 3; ++r)
      for (int q = 0; q < 3; ++q) S.M6[(3 + r) * 6 + q] = K[r * 3 + q];
  }
  __syncthreads();
  S.ok = sp.imu_mode == DRI_IMU_FIRST_ORDER
             ? preint_first_order(sp, c, S.x0.bg, S.x0.ba, S.W, S.P, S.fo)
             : preintegrate_block(sp.imu, S.x0.bg, S.x0.ba, false, 0.0, 0.0, S.W, S.P);
  if (!S.ok) return;
  imu_linearise(S.x0, S.x1, S.P, sp, S.L, S.J);
  // W_IMU = blockdiag(W_9, diag): W_9 J_a (columns 0..25) and W_9 e_a
  for (int idx = tid; idx < 9 * 26; idx += nt) {
    const int r = idx / 26, col = idx % 26;
    double acc = 0.0;
    for (int m = 0; m < 9; ++m) acc += c->Wimu[r * 18 + m] * S.J[m * 34 + col];
    S.WJa[idx] = acc;
  }
  if (tid >= 240 && tid < 249) {
    const int r = tid - 240;
    double acc = 0.0;
    for (int m = 0; m < 9; ++m) acc += c->Wimu[r * 18 + m] * S.L.e[m];
    S.We[r] = acc;
  }
  __syncthreads();
  // H upper from J_a^T W_9 J_a (the columns 0..25 it touches; the rest of the
  // upper triangle zero), b from -J_a^T W_9 e_a
  for (int idx = tid; idx < 26 * 26; idx += nt) {
    const int i = idx / 26, j = idx % 26;
    if (j < i) continue;
    double v = 0.0;
    for (int m = 0; m < 9; ++m) v += S.J[m * 34 + i] * S.WJa[m * 26 + j];
    S.H[i * 34 + j] = v;
  }
  for (int idx = tid; idx < 34 * 8; idx += nt) {
    const int i = idx / 8, j = 26 + idx % 8;
    if (j >= i) S.H[i * 34 + j] = 0.0;
  }
  if (tid >= 200 && tid < 200 + 34) {
    const int i = tid - 200;
    double v = 0.0;
    if (i < 26)
      for (int m = 0; m < 9; ++m) v -= S.J[m * 34 + i] * S.We[m];
    S.b[i] = v;
  }
  if (tid == 0) {
    double ce = 0.0;
    for (int m = 0; m < 9; ++m) ce += S.L.e[m] * S.We[m];
    for (int m = 9; m < 18; ++m) ce += S.L.e[m] * c->Wimu[m * 18 + m] * S.L.e[m];
    S.cost_imu = ce;
  }
  __syncthreads();
  // prior on x0: H00 += H*, b0 += b* - H* (x0 boxminus xbar)
  for (int idx = tid; idx < 17 * 17; idx += nt) {
    const int i = idx / 17, j = idx % 17;
    if (j >= i) S.H[i * 34 + j] += c->Hs[idx];
  }
  if (tid >= 192 && tid < 192 + 17) {
    const int i = tid - 192;
    double acc = c->bs[i];
    for (int k = 0; k < 17; ++k) acc -= c->Hs[i * 17 + k] * S.dprior[k];
    S.b[i] += acc;
  }
  __syncthreads();
  // Reduced system for the solve: x1's biases and gravity (columns 26..33) only
  // couple to x0's through the IMU's bias and gravity rows, so they are eliminated
  // in closed form.  The bias random walk then drops out exactly (x1's bias just
  // follows x0's) and the gravity rows leave w (A^T n)(n^T A), n the unit normal
  // of the range of x1's gravity block B: no cancellation of the 1e8-scale weights.
  for (int idx = tid; idx < 26 * 26; idx += nt) {
    const int i = idx / 26, j = idx % 26;
    S.Hr[idx] = j >= i ? S.H[i * 34 + j] : S.H[j * 34 + i];
  }
  if (tid < 26) S.br[tid] = S.b[tid];
  if (tid >= 32 && tid < 38) {
    const int k = (tid - 32) / 2, m = (tid - 32) % 2;
    S.Bg[tid - 32] = S.J[(15 + k) * 34 + 32 + m];
    S.Ag[tid - 32] = S.J[(15 + k) * 34 + 15 + m];
  }
  __syncthreads();
  if (tid == 0) {
    const double* B = S.Bg;   // B[k * 2 + m]
    double nv[3] = {B[2] * B[5] - B[4] * B[3], B[4] * B[1] - B[0] * B[5], B[0] * B[3] - B[2] * B[1]};
    const double inv = rsqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
    for (int i = 0; i < 3; ++i) nv[i] *= inv;
    const double w = c->Wimu[15 * 18 + 15];         // gravity weight (equal on its 3 rows)
    const double a0 = S.Ag[0] * nv[0] + S.Ag[2] * nv[1] + S.Ag[4] * nv[2];
    const double a1 = S.Ag[1] * nv[0] + S.Ag[3] * nv[1] + S.Ag[5] * nv[2];
    const double sn = nv[0] * S.L.e[15] + nv[1] * S.L.e[16] + nv[2] * S.L.e[17];
    S.Hr[15 * 26 + 15] += w * a0 * a0;
    S.Hr[15 * 26 + 16] += w * a0 * a1;
    S.Hr[16 * 26 + 15] += w * a0 * a1;
    S.Hr[16 * 26 + 16] += w * a1 * a1;
    S.br[15] -= w * a0 * sn;
    S.br[16] -= w * a1 * sn;
  }
  // full system (marginalisation, parity output): bias and gravity rows
  if (tid >= 32 && tid < 38) {          // bias rows 9..14: +I at x0, -I at x1
    const int i = tid - 32;
    const double w = c->Wimu[(9 + i) * 18 + 9 + i];
    S.H[(9 + i) * 34 + 9 + i] += w;
    S.H[(26 + i) * 34 + 26 + i] += w;
    S.H[(9 + i) * 34 + 26 + i] -= w;
    S.b[9 + i] -= w * S.L.e[9 + i];
    S.b[26 + i] += w * S.L.e[9 + i];
  } else if (tid >= 64 && tid < 74) {   // gravity rows 15..17, columns {15, 16, 32, 33}
    const int G[4] = {15, 16, 32, 33};
    int e = tid - 64, a = 0;
    while (e >= 4 - a) { e -= 4 - a; ++a; }
    const int ci = G[a], cj = G[a + e];
    double v = 0.0;
    for (int k = 0; k < 3; ++k)
      v += S.J[(15 + k) * 34 + ci] * c->Wimu[(15 + k) * 18 + 15 + k] * S.J[(15 + k) * 34 + cj];
    S.H[ci * 34 + cj] += v;
  } else if (tid >= 96 && tid < 100) {
    const int G[4] = {15, 16, 32, 33};
    const int ci = G[tid - 96];
    double v = 0.0;
    for (int k = 0; k < 3; ++k)
      v -= S.J[(15 + k) * 34 + ci] * c->Wimu[(15 + k) * 18 + 15 + k] * S.L.e[15 + k];
    S.b[ci] += v;
  }
  __syncthreads();
  if (sp.track_mode == DRI_TRACK_GYRO_ONLY) {
    // held components: identity rows and columns, zero right-hand side (their
    // step is zero; the reduced system is the leading 26 x 26 block of H).  No
    // pixel term touches them (they are not pose components).
    for (int idx = tid; idx < 34 * 34; idx += nt) {
      const int i = idx / 34, j = idx % 34;
      if (held_gyro_only(i) || held_gyro_only(j)) {
        const double v = i == j ? 1.0 : 0.0;
        if (j >= i) S.H[idx] = v;
        if (i < 26 && j < 26) S.Hr[i * 26 + j] = v;
      }
    }
    if (tid < 34 && held_gyro_only(tid)) {
      S.b[tid] = 0.0;
      if (tid < 26) S.br[tid] = 0.0;
    }
    __syncthreads();
  }
}

// The pixel terms after the pixel kernel (Eq. 3-4): the two 6x6 systems rotated
// into W (S.Hl, S.gl) and their contribution to the poses of x0 and x1, P12 and
// g12 in the order (x0 pose, x1 pose): the ICP term on x1's pose, the photometric
// term on both through B = [-M; I] (H12 = B H6 B^T).  128 threads (t = 0..127,
// four warps) that sync among themselves on named barrier BAR.
template <int BAR>
__device__ void pixel_terms(const SolveParams& sp, GnSmem& S, int t) {
  const Ctrl* c = sp.ctrl;
  if (t < 72) pixel_system_entry(sp, c, S, t);
  asm volatile("bar.sync %0, 128;" ::"n"(BAR) : "memory");
  if (t < 36) {                         // MH6 = M H6 (photometric term)
    const int i = t / 6, j = t % 6;
    double acc = 0.0;
    for (int k = 0; k < 6; ++k) acc += S.M6[i * 6 + k] * S.Hl[1][k * 6 + j];
    S.MH6[t] = acc;
  } else if (t >= 64 && t < 76) {       // g12: -M g6 on x0, g6 + g_icp on x1
    const int i = t - 64;
    if (i < 6) {
      double g0 = 0.0;
      for (int k = 0; k < 6; ++k) g0 -= S.M6[i * 6 + k] * S.gl[1][k];
      S.g12[i] = g0;
    } else {
      S.g12[i] = S.gl[1][i - 6] + S.gl[0][i - 6];
    }
  }
  asm volatile("bar.sync %0, 128;" ::"n"(BAR) : "memory");
  for (int idx = t; idx < 144; idx += 128) {
    const int i = idx / 12, j = idx % 12, a = i / 6, bb = j / 6, ii = i % 6, jj = j % 6;
    double v;
    if (a == 1 && bb == 1) {
      v = S.Hl[1][ii * 6 + jj] + S.Hl[0][ii * 6 + jj];
    } else if (a == 0 && bb == 1) {
      v = -S.MH6[ii * 6 + jj];
    } else if (a == 1 && bb == 0) {
      v = -S.MH6[jj * 6 + ii];
    } else {
      v = 0.0;
      for (int k = 0; k < 6; ++k) v += S.MH6[ii * 6 + k] * S.M6[jj * 6 + k];
    }
    S.P12[idx] = v;
  }
}

// Joint index of pose coordinate i (0..11) of (x0, x1).
__device__ __forceinline__ int pose_coord(int i) { return i < 6 ? i : 11 + i; }

// Adds P12, g12 to the upper triangle of S.H and to S.b (threads t0 .. t0 + n - 1).
__device__ void add_pixel_terms(GnSmem& S, int t, int n) {
  for (int idx = t; idx < 144; idx += n) {
    const int gi = pose_coord(idx / 12), gj = pose_coord(idx % 12);
    if (gj >= gi) S.H[gi * 34 + gj] += S.P12[idx];
  }
  if (t < 12) S.b[pose_coord(t)] += S.g12[t];
}

// The whole joint system at (ctrl->x0, ctrl->x1) into S.H (full) and S.b, with
// S.Hl, S.gl and S.cost_imu (dri_linearise).
__device__ void assemble(const SolveParams& sp, GnSmem& S) {
  const int tid = threadIdx.x, nt = blockDim.x;
  assemble_state(sp, S);
  if (!S.ok) return;
  grid_dep_wait();
  if (tid < 128) pixel_terms<3>(sp, S, tid);
  __syncthreads();
  add_pixel_terms(S, tid, nt);
  __syncthreads();
  for (int idx = tid; idx < 34 * 34; idx += nt) {
    const int i = idx / 34, j = idx % 34;
    if (j < i) S.H[idx] = S.H[j * 34 + i];
  }
  __syncthreads();
}

// RGB-D-only baseline (DRI_TRACK_RGBD_ONLY): one Gauss-Newton step on x1's pose
// with H_icp + lambda H_rgb (x1's blocks of the two pixel systems in W), x0
// fixed; 6x6 LDL^T; x1's other components unchanged.
__device__ void gn_step_pose_only(const SolveParams& sp, GnSmem& S) {
  Ctrl* c = sp.ctrl;
  const int tid = threadIdx.x;
  if (tid == 0) {
    S.x0 = c->x0;
    S.x1 = c->x1;
  }
  grid_dep_wait();                      // the pixel sums
  if (tid >= 32 && tid < 32 + 2 * 36) pixel_system_entry(sp, c, S, tid - 32);
  __syncthreads();
  const double lam = sp.rgbd_lambda;
  if (tid < 36) S.A[tid] = S.Hl[0][tid] + lam * S.Hl[1][tid];
  else if (tid < 42) S.x[tid - 36] = S.gl[0][tid - 36] + lam * S.gl[1][tid - 36];
  else if (tid < 53) S.x[tid - 36] = 0.0;                  // the other 11 tangent components
  __syncthreads();
  const bool pd = block_ldlt(S.A, 6, 6, S.col, &S.fail);
  if (tid == 0) ldlt_solve_thread(S.A, 6, 6, S.x);
  __syncthreads();
  bool good = pd;
  for (int i = 0; i < 6; ++i) good = good && isfinite(S.x[i]);
  if (!good) {
    if (tid == 0) c->status = DRI_ELOST;
    return;
  }
  const int warp = tid >> 5;
  if (warp == 0) {
    warp_state_boxplus(S.x1, S.x);
  } else if (tid == 64) {
    const double* s = c->sums;
    c->n_icp[sp.level] = (int32_t)s[28];
    c->n_rgb[sp.level] = (int32_t)s[kSums + 28];
    store_margin(c, sp.level);
    c->cost = sp.W_icp * s[27] + lam * sp.W_rgb * s[kSums + 27];
    c->iterations += 1;
  }
  __syncthreads();
  if (warp == 0) {
    warp_write_transforms(c, S.x0, S.x1, S.rot);
  } else if (tid == 32) {
    c->x1 = S.x1;
  }
}

// Solver order of the reduced system: the 14 components no pixel term touches
// (x0's velocity, biases and gravity, x1's velocity) first, then the 12 pose
// components of x0 and x1 in the order of P12.  Reduced index of solver index s.
__device__ __forceinline__ int solver_coord(int s) {
  return s < 11 ? 6 + s : (s < 14 ? 12 + s : (s < 20 ? s - 14 : s - 3));
}
constexpr int kNonPose = 14;

// One Gauss-Newton step of the joint problem (Eq. 7-8) on (x0, x1).  The
// state-only system is assembled and the sweep eliminates its 14 non-pose
// components before the pixel sums are read (they leave the Schur complement
// on the 12 pose components); warps 4-7 meanwhile wait for the pixel kernel
// and build the pixel terms, which warps 0-3 add to that complement before the
// last 12 pivots.  Jacobi scaling on the non-pose components (their diagonal
// is known before the pixel terms), none on the poses.
__device__ void gn_step_body(const SolveParams& sp, GnSmem& S) {
  Ctrl* c = sp.ctrl;
  if (c->status != 0) return;
  if (sp.track_mode == DRI_TRACK_RGBD_ONLY) {
    gn_step_pose_only(sp, S);
    return;
  }
  const int tid = threadIdx.x, nt = blockDim.x;
  assemble_state(sp, S);
  if (!S.ok) {
    if (tid == 0) c->status = DRI_ENOTREADY;
    return;
  }
  if (tid < 26) {
    const int k = solver_coord(tid);
    S.scale[tid] = tid < kNonPose ? rsqrt(fmax(S.Hr[k * 26 + k], 1e-300)) : 1.0;
  }
  __syncthreads();
  for (int idx = tid; idx < 26 * 26; idx += nt) {
    const int i = idx / 26, j = idx % 26;
    S.A[idx] = S.Hr[solver_coord(i) * 26 + solver_coord(j)] * S.scale[i] * S.scale[j];
  }
  if (tid < 26) S.xr[tid] = S.br[solver_coord(tid)] * S.scale[tid];
  __syncthreads();
  if (tid < 128) {
    const bool pd = ep_ldlt_solve<26, 128, kNonPose>(S.A, S.xr, S.xr, S.col, S.Lsm, S.piv, S.P12, S.g12);
    if (tid == 0) S.pd = pd;
  } else {
    grid_dep_wait();
    pixel_terms<3>(sp, S, tid - 128);
    asm volatile("bar.sync 2, 256;" ::: "memory");     // P12, g12 to the solver warps
    if (sp.last) add_pixel_terms(S, tid - 128, 128);
  }
  __syncthreads();
  if (tid < 26) S.x[solver_coord(tid)] = S.xr[tid] * S.scale[tid];
  __syncthreads();
  if (tid < 6) {
    S.x[26 + tid] = S.L.e[9 + tid] + S.x[9 + tid];          // x1 bias follows x0 bias
  } else if (tid == 32) {                                  // dg1 = -(B^T B)^-1 B^T (e_g + A dg0)
    const double* B = S.Bg;
    const double* A = S.Ag;
    double u[3];
    for (int k = 0; k < 3; ++k) u[k] = S.L.e[15 + k] + A[2 * k] * S.x[15] + A[2 * k + 1] * S.x[16];
    const double m00 = B[0] * B[0] + B[2] * B[2] + B[4] * B[4];
    const double m01 = B[0] * B[1] + B[2] * B[3] + B[4] * B[5];
    const double m11 = B[1] * B[1] + B[3] * B[3] + B[5] * B[5];
    const double q0 = B[0] * u[0] + B[2] * u[1] + B[4] * u[2];
    const double q1 = B[1] * u[0] + B[3] * u[1] + B[5] * u[2];
    const double idet = 1.0 / (m00 * m11 - m01 * m01);
    S.x[32] = -(m11 * q0 - m01 * q1) * idet;
    S.x[33] = -(m00 * q1 - m01 * q0) * idet;
  }
  __syncthreads();
  if (sp.track_mode == DRI_TRACK_GYRO_ONLY && tid < 34 && held_gyro_only(tid))
    S.x[tid] = 0.0;                                        // exactly zero, whatever e_g's rounding
  // every component finite (integer test of the exponent: no FP64 instruction)
  const bool fin = tid >= 34 || ((__double_as_longlong(S.x[tid]) >> 52) & 0x7ff) != 0x7ff;
  if (!__syncthreads_and(fin && S.pd)) {
    if (tid == 0) c->status = DRI_ELOST;
    return;
  }
  const int warp = tid >> 5;
  if (warp == 0) {
    warp_state_boxplus(S.x0, S.x);
  } else if (warp == 1) {
    warp_state_boxplus(S.x1, S.x + 17);
  } else if (tid == 64) {
    const double* s = c->sums;
    c->n_icp[sp.level] = (int32_t)s[28];
    c->n_rgb[sp.level] = (int32_t)s[kSums + 28];
    store_margin(c, sp.level);
    c->cost = sp.W_icp * s[27] + sp.W_rgb * s[kSums + 27] + S.cost_imu;
    c->iterations += 1;
  }
  __syncthreads();
  if (warp == 0) {
    warp_write_transforms(c, S.x0, S.x1, S.rot);
  } else if (tid == 32) {
    c->x0 = S.x0;
    c->x1 = S.x1;
  }
  if (sp.last) {
    for (int idx = tid; idx < 34 * 34; idx += nt) {
      const int i = idx / 34, j = idx % 34;
      c->H[idx] = j >= i ? S.H[idx] : S.H[j * 34 + i];
    }
    if (tid >= 64 && tid < 98) {
      c->b[tid - 64] = S.b[tid - 64];
      c->d[tid - 64] = S.x[tid - 64];
    }
  }
}

// ---------------------------------------------------------------------------
// 3-D gravity form (gravity_dof = DRI_GRAVITY_3D; Sec. II and IV-A keep q_IW
// with three degrees of freedom)
// ---------------------------------------------------------------------------
// The tangent space of a state has 18 dimensions (dr, da, dv, dbg, dba, dg with
// dg in R^3, q_IW <- exp(dg) (x) q_IW), the joint system 36.  The turn about
// gravity is a gauge that only the priors see, so each step is damped on the
// gravity components of both states: (H + mu D_g) dx = b, D_g the identity on
// coordinates 15..17 and 33..35, mu = kGravityDamping.  The damping regularises
// the step only: the cost, the reported system and the marginalisation use the
// undamped H.  The system is assembled whole (no closed-form elimination) and
// factorised by the element-parallel LDL^T at N = 36.
constexpr double kGravityDamping = 1.0;
constexpr int kNs3 = 18, kNj3 = 36;

__device__ __forceinline__ bool gravity_coord3(int k) { return (k >= 15 && k < 18) || k >= 33; }

struct Gn3Smem {
  ImuWork W;
  Preint P;
  ImuLin L;
  DState x0, x1;
  double J[18 * kNj3];
  double WJ[18 * kNj3];               // W_IMU J
  double We[18];                      // W_IMU e
  double H[kNj3 * kNj3];              // undamped joint system
  double A[kNj3 * kNj3];              // damped, Jacobi-scaled copy for the factorisation
  double b[kNj3], x[kNj3], scale[kNj3];
  double Hl[2][36];                   // world-frame 6x6 of ICP, photometric (weighted)
  double gl[2][6];
  double M6[36], MH6[36];
  double dprior[kNs3];
  double col[2 * (kNj3 + 1)];
  double Lsm[kNj3 * kNj3];
  double piv[kNj3];
  double fo[21];
  double rot[18];
  double cost_imu;
  int ok, pd;
};

// One Gauss-Newton step of the 3-D form (RGB-D-inertial tracking only).
__device__ void gn_step_g3(const SolveParams& sp, Gn3Smem& S) {
  Ctrl* c = sp.ctrl;
  if (c->status != 0) return;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) {
    S.x0 = c->x0;
    S.x1 = c->x1;
  }
  if ((tid >> 5) == 4) {
    warp_state_boxminus(c->x0, c->xbar, S.dprior, true);
  } else if (tid == 160) {
    for (int i = 0; i < 36; ++i) S.M6[i] = (i % 7 == 0) ? 1.0 : 0.0;
    const double d[3] = {c->x1.r[0] - c->x0.r[0], c->x1.r[1] - c->x0.r[1], c->x1.r[2] - c->x0.r[2]};
    double K[9];
    hat3(d, K);
    for (int r = 0; r < 3; ++r)
      for (int q = 0; q < 3; ++q) S.M6[(3 + r) * 6 + q] = K[r * 3 + q];
  }
  __syncthreads();
  S.ok = sp.imu_mode == DRI_IMU_FIRST_ORDER
             ? preint_first_order(sp, c, S.x0.bg, S.x0.ba, S.W, S.P, S.fo)
             : preintegrate_block(sp.imu, S.x0.bg, S.x0.ba, false, 0.0, 0.0, S.W, S.P);
  if (!S.ok) {
    if (tid == 0) c->status = DRI_ENOTREADY;
    return;
  }
  imu_linearise(S.x0, S.x1, S.P, sp, S.L, S.J, kNs3);
  for (int idx = tid; idx < 18 * kNj3; idx += nt) {
    const int r = idx / kNj3, col = idx % kNj3;
    double acc = 0.0;
    for (int m = 0; m < 18; ++m) acc += c->Wimu[r * 18 + m] * S.J[m * kNj3 + col];
    S.WJ[idx] = acc;
  }
  if (tid < 18) {
    double acc = 0.0;
    for (int m = 0; m < 18; ++m) acc += c->Wimu[tid * 18 + m] * S.L.e[m];
    S.We[tid] = acc;
  }
  // everything above depends on the states only; now the pixel sums
  grid_dep_wait();
  if (tid >= 32 && tid < 32 + 2 * 36) pixel_system_entry(sp, c, S, tid - 32);
  __syncthreads();
  if (tid < 36) {                       // MH6 = M H6 (photometric term)
    const int i = tid / 6, j = tid % 6;
    double acc = 0.0;
    for (int k = 0; k < 6; ++k) acc += S.M6[i * 6 + k] * S.Hl[1][k * 6 + j];
    S.MH6[tid] = acc;
  }
  // H upper = J^T W J, b = -J^T W e, the IMU cost
  for (int idx = tid; idx < kNj3 * kNj3; idx += nt) {
    const int i = idx / kNj3, j = idx % kNj3;
    if (j < i) continue;
    double v = 0.0;
    for (int m = 0; m < 18; ++m) v += S.J[m * kNj3 + i] * S.WJ[m * kNj3 + j];
    S.H[idx] = v;
  }
  if (tid >= 200 && tid < 200 + kNj3) {
    const int i = tid - 200;
    double v = 0.0;
    for (int m = 0; m < 18; ++m) v -= S.J[m * kNj3 + i] * S.We[m];
    S.b[i] = v;
  }
  if (tid == 0) {
    double ce = 0.0;
    for (int m = 0; m < 18; ++m) ce += S.L.e[m] * S.We[m];
    S.cost_imu = ce;
  }
  __syncthreads();
  // photometric on both poses (H12 = B H6 B^T, B = [-M; I]) and ICP on x1's pose
  for (int idx = tid; idx < 12 * 12; idx += nt) {
    const int i = idx / 12, j = idx % 12;
    if (j < i) continue;
    const int a = i / 6, bb = j / 6, ii = i % 6, jj = j % 6;
    double v;
    if (a == 1 && bb == 1) {
      v = S.Hl[1][ii * 6 + jj] + S.Hl[0][ii * 6 + jj];
    } else if (a == 0 && bb == 1) {
      v = -S.MH6[ii * 6 + jj];
    } else {
      v = 0.0;
      for (int k = 0; k < 6; ++k) v += S.MH6[ii * 6 + k] * S.M6[jj * 6 + k];
    }
    const int gi = a == 0 ? ii : kNs3 + ii, gj = bb == 0 ? jj : kNs3 + jj;
    S.H[gi * kNj3 + gj] += v;
  }
  if (tid >= 160 && tid < 166) {
    const int i = tid - 160;
    double g0 = 0.0;
    for (int k = 0; k < 6; ++k) g0 -= S.M6[i * 6 + k] * S.gl[1][k];
    S.b[i] += g0;
    S.b[kNs3 + i] += S.gl[1][i] + S.gl[0][i];
  }
  __syncthreads();
  // prior on x0: H00 += H*, b0 += b* - H* (x0 boxminus xbar)
  for (int idx = tid; idx < kNs3 * kNs3; idx += nt) {
    const int i = idx / kNs3, j = idx % kNs3;
    if (j >= i) S.H[i * kNj3 + j] += c->Hs[idx];
  }
  if (tid >= 192 && tid < 192 + kNs3) {
    const int i = tid - 192;
    double acc = c->bs[i];
    for (int k = 0; k < kNs3; ++k) acc -= c->Hs[i * kNs3 + k] * S.dprior[k];
    S.b[i] += acc;
  }
  __syncthreads();
  for (int idx = tid; idx < kNj3 * kNj3; idx += nt) {
    const int i = idx / kNj3, j = idx % kNj3;
    if (j < i) S.H[idx] = S.H[j * kNj3 + i];
  }
  __syncthreads();
  // the damped step, Jacobi-scaled
  if (tid < kNj3)
    S.scale[tid] = rsqrt(fmax(S.H[tid * kNj3 + tid] + (gravity_coord3(tid) ? kGravityDamping : 0.0), 1e-300));
  __syncthreads();
  for (int idx = tid; idx < kNj3 * kNj3; idx += nt) {
    const int i = idx / kNj3, j = idx % kNj3;
    const double h = S.H[idx] + ((i == j && gravity_coord3(i)) ? kGravityDamping : 0.0);
    S.A[idx] = h * S.scale[i] * S.scale[j];
  }
  if (tid < kNj3) S.x[tid] = S.b[tid] * S.scale[tid];
  __syncthreads();
  if (tid < 128) {
    const bool pd = ep_ldlt_solve<kNj3, 128>(S.A, S.x, S.x, S.col, S.Lsm, S.piv);
    if (tid == 0) S.pd = pd;
  }
  __syncthreads();
  if (tid < kNj3) S.x[tid] *= S.scale[tid];
  __syncthreads();
  bool good = S.pd;
  for (int i = 0; i < kNj3; ++i) good = good && isfinite(S.x[i]);
  if (!good) {
    if (tid == 0) c->status = DRI_ELOST;
    return;
  }
  const int warp = tid >> 5;
  if (warp == 0) {
    warp_state_boxplus(S.x0, S.x, true);
  } else if (warp == 1) {
    warp_state_boxplus(S.x1, S.x + kNs3, true);
  } else if (tid == 64) {
    const double* s = c->sums;
    c->n_icp[sp.level] = (int32_t)s[28];
    c->n_rgb[sp.level] = (int32_t)s[kSums + 28];
    store_margin(c, sp.level);
    c->cost = sp.W_icp * s[27] + sp.W_rgb * s[kSums + 27] + S.cost_imu;
    c->iterations += 1;
  }
  __syncthreads();
  if (warp == 0) {
    warp_write_transforms(c, S.x0, S.x1, S.rot);
  } else if (tid == 32) {
    c->x0 = S.x0;
    c->x1 = S.x1;
  }
  if (sp.last) {
    for (int idx = tid; idx < kNj3 * kNj3; idx += nt) c->H[idx] = S.H[idx];
    if (tid >= 64 && tid < 64 + kNj3) {
      c->b[tid - 64] = S.b[tid - 64];
      c->d[tid - 64] = S.x[tid - 64];
    }
  }
}

// W_IMU at c->x0 (noise propagated through the recursion, Sigma^-1), and the
// IMU prediction x^1(x0).  Whole block; false (status set) on failure.
struct BeginSmem {
  ImuWork W;
  Preint P;
  ImuLin L;
  double G[81], GS[81], Sg[81], Winv[81];
  double col[18];
  double rot[18];
  int ok, fail;
};

__device__ bool imu_weight_and_prediction(const SolveParams& sp, Ctrl* c, BeginSmem& B,
                                          DState* x1_pred) {
  const int tid = threadIdx.x;
  if (tid == 0) {
    B.ok = c->initialised && !(fabs(sp.imu->t0 - c->t_state) > 1e-9);
    if (!B.ok) c->status = DRI_ENOTREADY;
  }
  __syncthreads();
  if (!B.ok) return false;
  const DState x0 = c->x0;
  if (!preintegrate_block(sp.imu, x0.bg, x0.ba, true, sp.gyr_nd, sp.acc_nd, B.W, B.P)) {
    if (tid == 0) c->status = DRI_ENOTREADY;
    return false;
  }
  if (sp.imu_mode == DRI_IMU_FIRST_ORDER) store_lin(c, B.P, x0.bg, x0.ba);   // the frame's point
  imu_linearise(x0, x0, B.P, sp, B.L, nullptr);   // prediction only (x1 unused)
  // G = d(r^, a^, v^) / d(dphi, dv, dp)
  if (tid < 81) {
    const int r = tid / 9, q = tid % 9;
    double v = 0.0;
    if (r < 3 && q < 3) {              // [R^ rc]x RWS1
      double u[3];
      m3_vec(B.L.Rh, sp.r_CS, u);
      double K[9];
      hat3(u, K);
      v = K[r * 3] * B.L.RWS1[q] + K[r * 3 + 1] * B.L.RWS1[3 + q] + K[r * 3 + 2] * B.L.RWS1[6 + q];
    } else if (r < 3 && q >= 6) {
      v = B.L.A0[r * 3 + q - 6];
    } else if (r >= 3 && r < 6 && q < 3) {
      v = B.L.RWS1[(r - 3) * 3 + q];
    } else if (r >= 6 && q >= 3 && q < 6) {
      v = B.L.QA[(r - 6) * 3 + q - 3];
    }
    B.G[tid] = v;
  }
  __syncthreads();
  if (tid < 81) {
    const int r = tid / 9, q = tid % 9;
    double acc = 0.0;
    for (int k = 0; k < 9; ++k) acc += B.G[r * 9 + k] * B.P.Sig[k * 9 + q];
    B.GS[tid] = acc;
  }
  __syncthreads();
  if (tid < 81) {
    const int r = tid / 9, q = tid % 9;
    double acc = 0.0;
    for (int k = 0; k < 9; ++k) acc += B.GS[r * 9 + k] * B.G[q * 9 + k];
    B.Sg[tid] = acc;
  }
  __syncthreads();
  // gyro only: the rotation rows (3..5) keep the inverse of their own block
  // of the covariance; the position and velocity rows are dropped (identity
  // here, zero weight below)
  const bool gyro = sp.track_mode == DRI_TRACK_GYRO_ONLY;
  double sym = 0.0;
  if (tid < 81) {
    const int r = tid / 9, q = tid % 9;
    const bool rot = r >= 3 && r < 6 && q >= 3 && q < 6;
    sym = gyro && !rot ? (r == q ? 1.0 : 0.0) : 0.5 * (B.Sg[tid] + B.Sg[q * 9 + r]);
  }
  __syncthreads();
  if (tid < 81) B.Sg[tid] = sym;
  __syncthreads();
  const bool pd = block_ldlt(B.Sg, 9, 9, B.col, &B.fail);
  if (tid < 9) {
    double colv[9];
    for (int i = 0; i < 9; ++i) colv[i] = (i == tid) ? 1.0 : 0.0;
    ldlt_solve_thread(B.Sg, 9, 9, colv);
    for (int i = 0; i < 9; ++i) B.Winv[i * 9 + tid] = colv[i];
  }
  __syncthreads();
  for (int idx = tid; idx < 18 * 18; idx += blockDim.x) {
    const int r = idx / 18, q = idx % 18;
    double w = 0.0;
    if (r < 9 && q < 9) {
      if (!gyro || (r >= 3 && r < 6 && q >= 3 && q < 6)) w = 0.5 * (B.Winv[r * 9 + q] + B.Winv[q * 9 + r]);
    } else if (r == q) {
      if (r < 12) w = 1.0 / (sp.gyr_rw * sp.gyr_rw * B.P.T);
      else if (gyro) w = 0.0;                  // accelerometer bias and gravity rows
      else if (r < 15) w = 1.0 / (sp.acc_rw * sp.acc_rw * B.P.T);
      else w = 1.0 / (sp.sigma_grav * sp.sigma_grav);
    }
    c->Wimu[idx] = w;
  }
  if (tid == 0) {
    if (!pd) c->status = DRI_ELOST;
    if (x1_pred) {
      // x1 := x^1(x0): biases and q_IW carried over; gyro only: the predicted
      // rotation at x0's position and velocity
      DState x1 = x0;
      for (int i = 0; i < 3 && !gyro; ++i) {
        x1.r[i] = B.L.r[i];
        x1.v[i] = B.L.v[i];
      }
      rot_to_quat(B.L.Rh, x1.q);
      *x1_pred = x1;
    }
  }
  __syncthreads();
  return pd;
}

__device__ void frame_begin_body(const SolveParams& sp, BeginSmem& B) {
  Ctrl* c = sp.ctrl;
  const int tid = threadIdx.x;
  if (tid == 0) {
    c->status = 0;
    c->xstart = c->x;
    c->x0 = c->x;
    c->iterations = 0;
    c->cost = 0.0;
    for (int l = 0; l < kMaxLevels; ++l) c->n_icp[l] = c->n_rgb[l] = c->n_margin[l] = 0;
    c->margin_acc[0] = c->margin_acc[1] = 0u;
  }
  __syncthreads();
  if (sp.track_mode == DRI_TRACK_RGBD_ONLY) {     // x1 starts at x0; no IMU term
    if (tid == 0) {
      B.ok = c->initialised && !(fabs(sp.imu->t0 - c->t_state) > 1e-9);
      if (B.ok) c->x1 = c->x;
      else c->status = DRI_ENOTREADY;
    }
    __syncthreads();
    if (B.ok && (tid >> 5) == 0) warp_write_transforms(c, c->x0, c->x1, B.rot);
    return;
  }
  const bool ok = imu_weight_and_prediction(sp, c, B, &c->x1);
  if (ok && (tid >> 5) == 0) warp_write_transforms(c, c->x0, c->x1, B.rot);
}

// NS: tangent dimension of a state (17, or 18 for the 3-D gravity form).
template <int NS>
__device__ void frame_end_body(const SolveParams& sp) {
  constexpr int NJ = 2 * NS;
  Ctrl* c = sp.ctrl;
  const int tid = threadIdx.x;
  __shared__ int s_ok, s_fail;
  if (tid == 0) {
    if (c->status == 0 && c->n_icp[0] + c->n_rgb[0] < sp.min_valid) c->status = DRI_ELOST;
    s_ok = c->status == 0;
  }
  __syncthreads();
  if (!s_ok) {
    if (tid == 0) c->x = c->xstart;
    return;
  }
  if (sp.track_mode == DRI_TRACK_RGBD_ONLY) {     // no prior to carry over
    if (tid == 0) {
      c->x = c->x1;
      c->xbar = c->x1;
      c->t_state = sp.imu->t1;
      load_pose_ref(c);
      c->ref_index = 1 - c->ref_index;
    }
    return;
  }
  // b' = b - H d; Schur complement of the x0 block (Eq. 8)
  __shared__ double H[NJ * NJ];
  __shared__ double bp[NJ];
  __shared__ double L[NS * NS];
  __shared__ double X[NS * (NS + 1)];
  __shared__ double colbuf[NJ];
  __shared__ double Hs[NS * NS], bs[NS];
  for (int idx = tid; idx < NJ * NJ; idx += blockDim.x) H[idx] = c->H[idx];
  __syncthreads();
  if (tid < NJ) {
    double acc = c->b[tid];
    for (int k = 0; k < NJ; ++k) acc -= H[tid * NJ + k] * c->d[k];
    bp[tid] = acc;
  }
  for (int idx = tid; idx < NS * NS; idx += blockDim.x) L[idx] = H[(idx / NS) * NJ + idx % NS];
  __syncthreads();
  const bool pd = block_ldlt(L, NS, NS, colbuf, &s_fail);
  if (tid < NS + 1) {
    double colv[NS];
    for (int i = 0; i < NS; ++i) colv[i] = tid < NS ? H[i * NJ + NS + tid] : bp[i];
    ldlt_solve_thread(L, NS, NS, colv);
    for (int i = 0; i < NS; ++i) X[i * (NS + 1) + tid] = colv[i];
  }
  __syncthreads();
  for (int idx = tid; idx < NS * NS; idx += blockDim.x) {
    const int i = idx / NS, j = idx % NS;
    double acc = H[(NS + i) * NJ + NS + j];
    for (int k = 0; k < NS; ++k) acc -= H[(NS + i) * NJ + k] * X[k * (NS + 1) + j];
    Hs[idx] = acc;
  }
  if (tid < NS) {
    double acc = bp[NS + tid];
    for (int k = 0; k < NS; ++k) acc -= H[(NS + tid) * NJ + k] * X[k * (NS + 1) + NS];
    bs[tid] = acc;
  }
  __syncthreads();
  if (!pd) {
    if (tid == 0) {
      c->status = DRI_ELOST;
      c->x = c->xstart;
    }
    return;
  }
  // no information on held parts (gyro-only, 2-DoF form only)
  const bool gyro = NS == 17 && sp.track_mode == DRI_TRACK_GYRO_ONLY;
  for (int idx = tid; idx < NS * NS; idx += blockDim.x) {
    const int i = idx / NS, j = idx % NS;
    c->Hs[idx] = gyro && (held_gyro_only(i) || held_gyro_only(j)) ? 0.0 : 0.5 * (Hs[i * NS + j] + Hs[j * NS + i]);
  }
  if (tid < NS) c->bs[tid] = gyro && held_gyro_only(tid) ? 0.0 : bs[tid];
  if (tid == 0) {
    c->x = c->x1;
    c->xbar = c->x1;
    c->t_state = sp.imu->t1;
    load_pose_ref(c);
    c->ref_index = 1 - c->ref_index;
  }
}

template <int NS>
__device__ void frame_init_body(const SolveParams& sp) {
  const double t_frame = sp.imu->t1;
  Ctrl* c = sp.ctrl;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < NS * NS; idx += blockDim.x) {
    const int i = idx / NS, j = idx % NS;
    double v = 0.0;
    if (i == j) {
      const double s = i < 6 ? sp.prior_sigma[0]
                     : i < 9 ? sp.prior_sigma[1]
                     : i < 12 ? sp.prior_sigma[2]
                     : i < 15 ? sp.prior_sigma[3] : sp.prior_sigma[4];
      v = 1.0 / (s * s);
    }
    c->Hs[idx] = v;
  }
  if (tid < NS) c->bs[tid] = 0.0;
  if (tid == 0) {
    c->status = 0;
    c->xbar = c->x;
    c->x0 = c->x;
    c->x1 = c->x;
    c->xstart = c->x;
    c->t_state = t_frame;
    load_pose_ref(c);
    c->ref_index = 1 - c->ref_index;
    c->initialised = 1;
    c->iterations = 0;
    c->cost = 0.0;
    for (int l = 0; l < kMaxLevels; ++l) c->n_icp[l] = c->n_rgb[l] = c->n_margin[l] = 0;
    c->margin_acc[0] = c->margin_acc[1] = 0u;
  }
}

__global__ void __launch_bounds__(kSolveThreads) k_linearise_begin(SolveParams sp, DState x0, DState x1) {
  Ctrl* c = sp.ctrl;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BeginSmem& B = *reinterpret_cast<BeginSmem*>(smem_raw);
  const int tid = threadIdx.x;
  if (tid == 0) {
    c->status = 0;
    c->x0 = x0;
    c->x1 = x1;
    c->margin_acc[0] = c->margin_acc[1] = 0u;
  }
  __syncthreads();
  const bool ok = imu_weight_and_prediction(sp, c, B, nullptr);
  if (ok && (tid >> 5) == 0) warp_write_transforms(c, c->x0, c->x1, B.rot);
}

__global__ void __launch_bounds__(kSolveThreads) k_linearise_end(SolveParams sp, dri_linearisation* out) {
  Ctrl* c = sp.ctrl;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  GnSmem& S = *reinterpret_cast<GnSmem*>(smem_raw);
  assemble(sp, S);
  const int tid = threadIdx.x;
  for (int idx = tid; idx < 34 * 34; idx += blockDim.x) out->H[idx] = S.ok ? S.H[idx] : 0.0;
  if (tid < 34) out->b[tid] = S.ok ? S.b[tid] : 0.0;
  if (tid < 36) {
    out->H_icp[tid] = S.Hl[0][tid];
    out->H_rgb[tid] = S.Hl[1][tid];
  }
  if (tid < 6) {
    out->b_icp[tid] = S.gl[0][tid];
    out->b_rgb[tid] = S.gl[1][tid];
  }
  if (tid < 18) out->e_imu[tid] = S.ok ? S.L.e[tid] : 0.0;
  if (tid == 0) {
    const double* s = c->sums;
    out->cost_icp = sp.W_icp * s[27];
    out->cost_rgb = sp.W_rgb * s[kSums + 27];
    out->cost_imu = S.ok ? S.cost_imu : 0.0;
    out->n_icp = (int64_t)s[28];
    out->n_rgb = (int64_t)s[kSums + 28];
    out->n_margin_icp = c->margin_acc[0];
    out->n_margin_rgb = c->margin_acc[1];
    c->margin_acc[0] = c->margin_acc[1] = 0u;
    if (!S.ok) c->status = DRI_ENOTREADY;
  }
}

// Slot blockIdx.x of a batched launch: its SolveParams with this launch's IMU
// block, level and last-iteration flag, copied to shared memory; returns the
// slot's mode (uniform over the block).
__device__ int load_slot_params(const BatchArgs& a, SolveParams& sp) {
  const int slot = a.slot0 + blockIdx.x;
  const SlotDyn& d = batch_dyn(a, slot);
  const int mode = d.mode;
  if (mode == kSlotIdle) return mode;
  const uint32_t* src = reinterpret_cast<const uint32_t*>(&a.slots[slot].sp);
  uint32_t* dst = reinterpret_cast<uint32_t*>(&sp);
  for (int i = threadIdx.x; i < (int)(sizeof(SolveParams) / 4); i += blockDim.x) dst[i] = src[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    sp.imu = reinterpret_cast<const ImuHeader*>(a.dyn + d.imu_off);
    sp.level = a.level;
    sp.last = a.last;
  }
  __syncthreads();
  return mode;
}

// One block per slot: a tracked slot starts its frame (x0 := x, IMU weight and
// prediction), an initialising slot takes the first-frame prior.
__global__ void __launch_bounds__(kSolveThreads) k_frame_begin_batch(const BatchArgs a) {
  __shared__ SolveParams sp;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (load_slot_params(a, sp) == kSlotTrack) frame_begin_body(sp, *reinterpret_cast<BeginSmem*>(smem_raw));
}

constexpr size_t kGnSmemMax = sizeof(Gn3Smem) > sizeof(GnSmem) ? sizeof(Gn3Smem) : sizeof(GnSmem);

__global__ void __launch_bounds__(kSolveThreads) k_gn_step_batch(const BatchArgs a) {
  __shared__ SolveParams sp;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  grid_dep_launch();                    // the next pixel kernel waits for this step itself
  const int mode = load_slot_params(a, sp);
  if (mode == kSlotTrack && sp.gdof == 3) gn_step_g3(sp, *reinterpret_cast<Gn3Smem*>(smem_raw));
  else if (mode == kSlotTrack) gn_step_body(sp, *reinterpret_cast<GnSmem*>(smem_raw));
  else grid_dep_wait();                 // idle slot: nothing to read, keep the ordering
}

// A first frame is initialised here too, so that the map sets of every slot
// swap only at the frame end: the map kernels of the frame, which may run
// beside its start, read which set is the reference.
__global__ void __launch_bounds__(kSolveThreads) k_frame_end_batch(const BatchArgs a) {
  __shared__ SolveParams sp;
  const int mode = load_slot_params(a, sp);
  if (mode == kSlotTrack) {
    if (sp.gdof == 3) frame_end_body<18>(sp);
    else frame_end_body<17>(sp);
  } else if (mode == kSlotInit) {
    if (sp.gdof == 3) frame_init_body<18>(sp);
    else frame_init_body<17>(sp);
  }
}

// Result heads of all slots into one contiguous buffer (one copy to the host).
__global__ void k_gather_heads(const BatchArgs a, unsigned char* __restrict__ out) {
  const int slot = a.slot0 + blockIdx.x;
  const uint64_t* src = reinterpret_cast<const uint64_t*>(a.slots[slot].sp.ctrl);
  uint64_t* dst = reinterpret_cast<uint64_t*>(out + (size_t)slot * kCtrlHeadBytes);
  for (int i = threadIdx.x; i < (int)(kCtrlHeadBytes / 8); i += blockDim.x) dst[i] = src[i];
}

}  // namespace

cudaError_t prepare_solver_kernels() {
  cudaError_t e = cudaFuncSetAttribute(k_gn_step_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kGnSmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_linearise_end, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(GnSmem));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_frame_begin_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(BeginSmem));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_linearise_begin, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(BeginSmem));
  return e;
}

int solver_max_imu_pieces() { return kMaxPieces; }

cudaError_t launch_frame_begin_batch(const BatchArgs& a, cudaStream_t s) {
  k_frame_begin_batch<<<a.nslots, kSolveThreads, sizeof(BeginSmem), s>>>(a);
  return cudaGetLastError();
}
int launch_priority(bool solver) {
  static const int2 range = [] {
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) least = greatest = 0;
    return make_int2(least, greatest);
  }();
  // greater priority is the numerically smaller value
  const int p = solver ? range.y : range.y + 1;
  return p < range.x ? p : range.x;
}

// The step's blocks are scheduled ahead of pixel-kernel blocks waiting for an
// SM: with several slot groups, one group's FP64 step runs beside another
// group's pixel kernel instead of waiting for its last wave.

cudaError_t launch_gn_step_batch(const BatchArgs& a, bool g3, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(a.nslots);
  cfg.blockDim = dim3(kSolveThreads);
  cfg.dynamicSmemBytes = g3 ? kGnSmemMax : sizeof(GnSmem);
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  attr[1].id = cudaLaunchAttributePriority;
  attr[1].val.priority = launch_priority(true);
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, k_gn_step_batch, a);
}
cudaError_t launch_frame_end_batch(const BatchArgs& a, cudaStream_t s) {
  k_frame_end_batch<<<a.nslots, kSolveThreads, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_gather_heads(const BatchArgs& a, unsigned char* out, cudaStream_t s) {
  k_gather_heads<<<a.nslots, 64, 0, s>>>(a, out);
  return cudaGetLastError();
}
cudaError_t launch_linearise_begin(const SolveParams& p, const DState& x0, const DState& x1,
                                   cudaStream_t s) {
  k_linearise_begin<<<1, kSolveThreads, sizeof(BeginSmem), s>>>(p, x0, x1);
  return cudaGetLastError();
}
cudaError_t launch_linearise_end(const SolveParams& p, dri_linearisation* out, cudaStream_t s) {
  k_linearise_end<<<1, kSolveThreads, sizeof(GnSmem), s>>>(p, out);
  return cudaGetLastError();
}

}  // namespace dri
