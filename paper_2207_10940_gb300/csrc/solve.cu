// FP64 single-block solver kernels of the tracking loop (Sec. IV-C/D/E).
//
//   frame_begin   x0 := x; IMU pre-integration at x0's biases with the propagated
//                 noise covariance; W_IMU = Sigma^-1; x1 := the IMU prediction x^1(x0)
//   gn_step       one Gauss-Newton iteration: re-integrate the IMU at x0's current
//                 biases, IMU error (Eq. 5) and its analytic 18x34 Jacobian; rotate
//                 the pixel kernel's photometric / ICP systems into W and map the
//                 photometric one onto both poses; add the prior (Eq. 6/9); solve the
//                 34x34 system of Eq. 7 by Cholesky; x0, x1 boxplus= dx (Eq. 2)
//   frame_end     marginalise x0 by the Schur complement (Eq. 8) at the updated point,
//                 make the frame the reference (flip of the map sets)
//   frame_init    first frame: first-frame prior, the frame becomes the reference
//
// Readings (the paper gives no integration scheme, Jacobians or prior sign):
// zero-order-hold integration cut at sample times, update order p, v, R; the bias
// Jacobians are the exact derivatives of that recursion; W_IMU is block diagonal
// (propagated (r, a, v) block, bias random walks, gravity noise) and fixed per
// frame; the prior adds H* to H_00 and b* - H* (x0 boxminus xbar) to b_0; after the
// last update b <- b - H dx before the Schur complement.
//
// All arithmetic here is FP64.  One block of kSolveThreads threads runs each kernel.
#include <cmath>

#include "dri_internal.h"
#include "so3.cuh"

namespace dri {

namespace {

constexpr int kSolveThreads = 256;
constexpr int kMaxPieces = 256;

struct Preint {
  double dR[9], dv[3], dp[3];
  double Phig[9], Vg[9], Pg[9], Va[9], Pa[9];
  double Sig[81];
  double T;
};

struct Pred {
  double r[3], R[9], v[3], c[3];
  double RWS1[9];       // R_WC0 R_CS dR
  double A0[9];         // R_WC0 R_CS
  double R0[9], Q0[9];
};

__device__ __forceinline__ const dri_imu_sample* imu_samples(const ImuHeader* h) {
  return reinterpret_cast<const dri_imu_sample*>(h + 1);
}

// Zero-order-hold pieces of [t0, t1]: sample index and duration.  -1 if the
// samples do not cover the interval.
__device__ int imu_pieces(const ImuHeader* h, int* pk, double* pdt) {
  const dri_imu_sample* s = imu_samples(h);
  const int n = h->n;
  const double t0 = h->t0, t1 = h->t1;
  if (n <= 0 || s[0].t > t0 || s[n - 1].t < t1 || !(t1 > t0)) return -1;
  int k = 0;
  while (k + 1 < n && s[k + 1].t <= t0) ++k;
  double tau = t0;
  int np = 0;
  while (tau < t1) {
    const double nxt = (k + 1 >= n) ? t1 : fmin(s[k + 1].t, t1);
    if (nxt > tau) {
      if (np >= kMaxPieces) return -1;
      pk[np] = k;
      pdt[np] = nxt - tau;
      ++np;
    }
    tau = nxt;
    ++k;
  }
  return np;
}

// Sequential pre-integration with bias Jacobians (and noise covariance if cov).
__device__ void preintegrate(const ImuHeader* h, const int* pk, const double* pdt, int np,
                             const double* bg, const double* ba, bool cov, double gnd, double and_,
                             Preint& P) {
  const dri_imu_sample* s = imu_samples(h);
  for (int i = 0; i < 9; ++i) {
    P.dR[i] = (i % 4 == 0) ? 1.0 : 0.0;
    P.Phig[i] = P.Vg[i] = P.Pg[i] = P.Va[i] = P.Pa[i] = 0.0;
  }
  for (int i = 0; i < 3; ++i) P.dv[i] = P.dp[i] = 0.0;
  if (cov)
    for (int i = 0; i < 81; ++i) P.Sig[i] = 0.0;
  double T = 0.0;
  for (int j = 0; j < np; ++j) {
    const dri_imu_sample& m = s[pk[j]];
    const double dt = pdt[j];
    T += dt;
    const double w[3] = {m.gyr[0] - bg[0], m.gyr[1] - bg[1], m.gyr[2] - bg[2]};
    const double a[3] = {m.acc[0] - ba[0], m.acc[1] - ba[1], m.acc[2] - ba[2]};
    const double th[3] = {w[0] * dt, w[1] * dt, w[2] * dt};
    double E[9], Jr[9], K[9], Ah[9], t1[9], t2[9];
    so3_exp(th, E);
    so3_jr(th, Jr);
    hat3(a, K);
    m3_mul(P.dR, K, Ah);  // dR [a]x
    // bias Jacobians of the recursion (old values on the right-hand side)
    m3_mul(Ah, P.Phig, t1);  // dR [a]x Phi_g
    for (int i = 0; i < 9; ++i) {
      P.Pg[i] += P.Vg[i] * dt - 0.5 * t1[i] * dt * dt;
      P.Pa[i] += P.Va[i] * dt - 0.5 * P.dR[i] * dt * dt;
      P.Vg[i] -= t1[i] * dt;
      P.Va[i] -= P.dR[i] * dt;
    }
    m3_tmul(E, P.Phig, t2);  // E^T Phi_g
    for (int i = 0; i < 9; ++i) P.Phig[i] = t2[i] - Jr[i] * dt;
    if (cov) {
      // Sigma <- A Sigma A^T + Bg (gnd^2/dt) Bg^T + Ba (and^2/dt) Ba^T, order (phi, v, p)
      double A[81];
      for (int i = 0; i < 81; ++i) A[i] = 0.0;
      for (int i = 0; i < 9; ++i) A[i * 9 + i] = 1.0;
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
          A[r * 9 + c] = E[c * 3 + r];                              // E^T
          A[(3 + r) * 9 + c] = -Ah[r * 3 + c] * dt;
          A[(6 + r) * 9 + c] = -0.5 * Ah[r * 3 + c] * dt * dt;
        }
      for (int r = 0; r < 3; ++r) A[(6 + r) * 9 + 3 + r] = dt;
      double AS[81];
      for (int r = 0; r < 9; ++r)
        for (int c = 0; c < 9; ++c) {
          double acc = 0.0;
          for (int k = 0; k < 9; ++k) acc += A[r * 9 + k] * P.Sig[k * 9 + c];
          AS[r * 9 + c] = acc;
        }
      double B[27];   // Bg columns 0..2 scaled, Ba columns in a second pass
      const double qg = gnd * gnd / dt, qa = and_ * and_ / dt;
      for (int r = 0; r < 9; ++r)
        for (int c = r; c < 9; ++c) {
          double acc = 0.0;
          for (int k = 0; k < 9; ++k) acc += AS[r * 9 + k] * A[c * 9 + k];
          P.Sig[r * 9 + c] = acc;
        }
      // Bg = [Jr dt; 0; 0]
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) B[r * 3 + c] = Jr[r * 3 + c] * dt;
      for (int r = 0; r < 3; ++r)
        for (int c = r; c < 3; ++c) {
          double acc = 0.0;
          for (int k = 0; k < 3; ++k) acc += B[r * 3 + k] * B[c * 3 + k];
          P.Sig[r * 9 + c] += qg * acc;
        }
      // Ba = [0; dR dt; 0.5 dR dt^2]
      double Bv[9], Bp[9];
      for (int i = 0; i < 9; ++i) {
        Bv[i] = P.dR[i] * dt;
        Bp[i] = 0.5 * P.dR[i] * dt * dt;
      }
      for (int r = 0; r < 6; ++r)
        for (int c = r; c < 6; ++c) {
          const double* Br = r < 3 ? Bv + 3 * r : Bp + 3 * (r - 3);
          const double* Bc = c < 3 ? Bv + 3 * c : Bp + 3 * (c - 3);
          P.Sig[(3 + r) * 9 + 3 + c] += qa * (Br[0] * Bc[0] + Br[1] * Bc[1] + Br[2] * Bc[2]);
        }
      for (int r = 0; r < 9; ++r)
        for (int c = 0; c < r; ++c) P.Sig[r * 9 + c] = P.Sig[c * 9 + r];
    }
    // state recursion: p, then v, then R
    double Ra[3];
    m3_vec(P.dR, a, Ra);
    for (int i = 0; i < 3; ++i) {
      P.dp[i] += P.dv[i] * dt + 0.5 * Ra[i] * dt * dt;
      P.dv[i] += Ra[i] * dt;
    }
    m3_mul(P.dR, E, t1);
    for (int i = 0; i < 9; ++i) P.dR[i] = t1[i];
  }
  P.T = T;
}

__device__ void predict(const DState& x0, const Preint& P, const SolveParams& sp, Pred& o) {
  quat_to_rot(x0.q, o.R0);
  quat_to_rot(x0.qg, o.Q0);
  m3_mul(o.R0, sp.R_CS, o.A0);
  m3_mul(o.A0, P.dR, o.RWS1);
  m3_mult(o.RWS1, sp.R_CS, o.R);                 // R^ = R0 Rc dR Rc^T
  const double T = P.T;
  const double gI[3] = {0.0, 0.0, -sp.g};
  for (int i = 0; i < 3; ++i) o.c[i] = x0.v[i] * T + 0.5 * gI[i] * T * T;
  double t1[3], t2[3], t3[3], t4[3];
  m3_vec(o.R0, sp.r_CS, t1);
  m3_tvec(o.Q0, o.c, t2);
  m3_vec(o.A0, P.dp, t3);
  m3_vec(o.R, sp.r_CS, t4);
  for (int i = 0; i < 3; ++i) o.r[i] = x0.r[i] + t1[i] + t2[i] + t3[i] - t4[i];
  double QA[9], t5[3];
  m3_mul(o.Q0, o.A0, QA);
  m3_vec(QA, P.dv, t5);
  for (int i = 0; i < 3; ++i) o.v[i] = x0.v[i] + gI[i] * T + t5[i];
}

// e = x^1(x0) boxminus x1 (18) and de/d(dx0, dx1) (18 x 34, row-major).
__device__ void imu_error_jacobian(const DState& x0, const DState& x1, const Preint& P,
                                   const Pred& pr, const SolveParams& sp, double* e, double* J) {
  double R1[9], Q1[9], M[9], t[9];
  quat_to_rot(x1.q, R1);
  quat_to_rot(x1.qg, Q1);
  for (int i = 0; i < 3; ++i) e[i] = pr.r[i] - x1.r[i];
  m3_mult(pr.R, R1, M);
  so3_log(M, e + 3);
  for (int i = 0; i < 3; ++i) {
    e[6 + i] = pr.v[i] - x1.v[i];
    e[9 + i] = x0.bg[i] - x1.bg[i];
    e[12 + i] = x0.ba[i] - x1.ba[i];
  }
  m3_mult(pr.Q0, Q1, M);
  so3_log(M, e + 15);
  if (J == nullptr) return;
  for (int i = 0; i < 18 * 34; ++i) J[i] = 0.0;
  auto put3 = [&](int r0, int c0, const double* B) {
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) J[(r0 + r) * 34 + c0 + c] = B[r * 3 + c];
  };
  auto put32 = [&](int r0, int c0, const double* B) {   // B (3x3) times P2 = first two columns
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 2; ++c) J[(r0 + r) * 34 + c0 + c] = B[r * 3 + c];
  };
  auto ident = [&](int r0, int c0, double s) {
    for (int r = 0; r < 3; ++r) J[(r0 + r) * 34 + c0 + r] = s;
  };
  double Jla[9], Jlg[9], Jra[9], Jrg[9];
  so3_jl_inv(e + 3, Jla);
  so3_jl_inv(e + 15, Jlg);
  so3_jr_inv(e + 3, Jra);
  so3_jr_inv(e + 15, Jrg);
  // x1 columns 17..33
  ident(0, 17, -1.0);
  for (int i = 0; i < 9; ++i) t[i] = -Jra[i];
  put3(3, 20, t);
  ident(6, 23, -1.0);
  ident(9, 26, -1.0);
  ident(12, 29, -1.0);
  for (int i = 0; i < 9; ++i) t[i] = -Jrg[i];
  put32(15, 32, t);
  // x0 columns 0..16
  ident(0, 0, 1.0);
  {
    double u[3], QTc[3];
    m3_tvec(pr.Q0, pr.c, QTc);
    for (int i = 0; i < 3; ++i) u[i] = -(pr.r[i] - x0.r[i] - QTc[i]);
    hat3(u, t);
    put3(0, 3, t);                                   // -[r^ - r0 - Q0^T c]x
  }
  put3(3, 3, Jla);
  double Adv[3], K[9], QK[9];
  m3_vec(pr.A0, P.dv, Adv);
  hat3(Adv, K);
  m3_mul(pr.Q0, K, QK);
  for (int i = 0; i < 9; ++i) t[i] = -QK[i];
  put3(6, 3, t);                                     // -Q0 [A0 dv]x
  for (int i = 0; i < 9; ++i) t[i] = pr.Q0[(i % 3) * 3 + i / 3] * P.T;
  put3(0, 6, t);                                     // Q0^T T
  ident(6, 6, 1.0);
  {
    double Rrc[3], Kr[9], KR[9], KRP[9], AP[9];
    m3_vec(pr.R, sp.r_CS, Rrc);
    hat3(Rrc, Kr);
    m3_mul(Kr, pr.RWS1, KR);
    m3_mul(KR, P.Phig, KRP);
    m3_mul(pr.A0, P.Pg, AP);
    for (int i = 0; i < 9; ++i) t[i] = AP[i] + KRP[i];
    put3(0, 9, t);                                   // A0 Pg + [R^ rc]x RWS1 Phig
    double RP[9];
    m3_mul(pr.RWS1, P.Phig, RP);
    m3_mul(Jla, RP, t);
    put3(3, 9, t);                                   // Jl^-1(e_a) RWS1 Phig
    double QA[9];
    m3_mul(pr.Q0, pr.A0, QA);
    m3_mul(QA, P.Vg, t);
    put3(6, 9, t);                                   // Q0 A0 Vg
    ident(9, 9, 1.0);
    m3_mul(pr.A0, P.Pa, t);
    put3(0, 12, t);                                  // A0 Pa
    m3_mul(QA, P.Va, t);
    put3(6, 12, t);                                  // Q0 A0 Va
    ident(12, 12, 1.0);
    double Kc[9];
    hat3(pr.c, Kc);
    m3_tmul(pr.Q0, Kc, t);
    put32(0, 15, t);                                 // Q0^T [c]x P2
    double QAdv[3];
    m3_vec(QA, P.dv, QAdv);
    hat3(QAdv, Kc);
    for (int i = 0; i < 9; ++i) t[i] = -Kc[i];
    put32(6, 15, t);                                 // -[Q0 A0 dv]x P2
    put32(15, 15, Jlg);                              // Jl^-1(e_g) P2
  }
}

// x boxminus y (17): vector parts subtract, orientations log(p q^-1), gravity x, y of its log.
__device__ void state_boxminus(const DState& x, const DState& y, double* d) {
  double Rx[9], Ry[9], M[9], w[3];
  for (int i = 0; i < 3; ++i) {
    d[i] = x.r[i] - y.r[i];
    d[6 + i] = x.v[i] - y.v[i];
    d[9 + i] = x.bg[i] - y.bg[i];
    d[12 + i] = x.ba[i] - y.ba[i];
  }
  quat_to_rot(x.q, Rx);
  quat_to_rot(y.q, Ry);
  m3_mult(Rx, Ry, M);
  so3_log(M, d + 3);
  quat_to_rot(x.qg, Rx);
  quat_to_rot(y.qg, Ry);
  m3_mult(Rx, Ry, M);
  so3_log(M, w);
  d[15] = w[0];
  d[16] = w[1];
}

__device__ void state_boxplus(DState& x, const double* d) {
  for (int i = 0; i < 3; ++i) {
    x.r[i] += d[i];
    x.v[i] += d[6 + i];
    x.bg[i] += d[9 + i];
    x.ba[i] += d[12 + i];
  }
  quat_boxplus(x.q, d + 3);
  const double dg[3] = {d[15], d[16], 0.0};
  quat_boxplus(x.qg, dg);
}

// Pixel-kernel transforms for the next linearisation (FP64 -> FP32 once).
__device__ void write_transforms(Ctrl* c) {
  double R0[9], R1[9], M[9], dr[3], t[3];
  quat_to_rot(c->x0.q, R0);
  quat_to_rot(c->x1.q, R1);
  m3_tmul(c->Rref, R1, M);
  for (int i = 0; i < 3; ++i) dr[i] = c->x1.r[i] - c->rref[i];
  m3_tvec(c->Rref, dr, t);
  for (int i = 0; i < 9; ++i) c->xf_icp[i] = (float)(M[i] - ((i % 4 == 0) ? 1.0 : 0.0));
  for (int i = 0; i < 3; ++i) c->xf_icp[9 + i] = (float)t[i];
  m3_tmul(R0, R1, M);
  for (int i = 0; i < 3; ++i) dr[i] = c->x1.r[i] - c->x0.r[i];
  m3_tvec(R0, dr, t);
  for (int i = 0; i < 9; ++i) c->xf_rgb[i] = (float)(M[i] - ((i % 4 == 0) ? 1.0 : 0.0));
  for (int i = 0; i < 3; ++i) c->xf_rgb[9 + i] = (float)t[i];
}

// In-place Cholesky A = L L^T (lower triangle), whole block; false if not positive definite.
__device__ bool block_cholesky(double* A, int n, int ld) {
  __shared__ int s_fail;
  if (threadIdx.x == 0) s_fail = 0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      double a = A[k * ld + k];
      if (!(a > 0.0) || !isfinite(a)) {
        s_fail = 1;
        a = 1.0;
      }
      A[k * ld + k] = sqrt(a);
    }
    __syncthreads();
    const double piv = A[k * ld + k];
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) A[i * ld + k] /= piv;
    __syncthreads();
    const int m = n - k - 1;
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
      const int i = k + 1 + idx / m, j = k + 1 + idx % m;
      if (j <= i) A[i * ld + j] -= A[i * ld + k] * A[j * ld + k];
    }
    __syncthreads();
  }
  return s_fail == 0;
}

// Solve L L^T x = b in place on b (thread 0; n <= 64).
__device__ void chol_subst(const double* L, int n, int ld, double* b) {
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= L[i * ld + k] * b[k];
    b[i] = s / L[i * ld + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int k = i + 1; k < n; ++k) s -= L[k * ld + i] * b[k];
    b[i] = s / L[i * ld + i];
  }
}

struct StepShared {
  double H[34 * 34];
  double b[34];
  double J[18 * 34];
  double WJ[18 * 34];
  double e[18];
  double Hl[2][36];          // world-frame 6x6 of ICP, photometric (weighted)
  double gl[2][6];           // weighted b of each term (x1 pose)
  double M6[36];             // [[I,0],[[r1-r0]x, I]]
  double scale[34];
  double cost_imu;
  int pk[kMaxPieces];
  double pdt[kMaxPieces];
  int np;
  int ok;
};

// Assemble the joint system of Eq. 7 at (ctrl->x0, ctrl->x1) in shared memory.
__device__ void assemble(const SolveParams& sp, StepShared& S) {
  Ctrl* c = sp.ctrl;
  const int tid = threadIdx.x;
  __shared__ Preint s_pre;
  __shared__ Pred s_pred;
  if (tid == 0) {
    S.np = imu_pieces(sp.imu, S.pk, S.pdt);
    S.ok = S.np > 0;
    if (S.ok) {
      preintegrate(sp.imu, S.pk, S.pdt, S.np, c->x0.bg, c->x0.ba, false, 0.0, 0.0, s_pre);
      predict(c->x0, s_pre, sp, s_pred);
      imu_error_jacobian(c->x0, c->x1, s_pre, s_pred, sp, S.e, S.J);
    }
  }
  // meanwhile: pixel systems into W (term 0 ICP with R_ref, term 1 photometric with R_0)
  if (tid >= 32 && tid < 32 + 2 * 36) {
    const int term = (tid - 32) / 36, idx = (tid - 32) % 36;
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
    // Hw = Q Hloc Q^T with Q = diag(R, R): Hw_ij = sum_kl Q_ik Hloc_kl Q_jl
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
  __syncthreads();
  if (!S.ok) return;
  // WJ = W_imu J
  for (int idx = tid; idx < 18 * 34; idx += blockDim.x) {
    const int r = idx / 34, col = idx % 34;
    double acc = 0.0;
    for (int k = 0; k < 18; ++k) acc += c->Wimu[r * 18 + k] * S.J[k * 34 + col];
    S.WJ[idx] = acc;
  }
  if (tid == 0) {
    for (int i = 0; i < 36; ++i) S.M6[i] = (i % 7 == 0) ? 1.0 : 0.0;
    const double d[3] = {c->x1.r[0] - c->x0.r[0], c->x1.r[1] - c->x0.r[1], c->x1.r[2] - c->x0.r[2]};
    double K[9];
    hat3(d, K);
    for (int r = 0; r < 3; ++r)
      for (int q = 0; q < 3; ++q) S.M6[(3 + r) * 6 + q] = K[r * 3 + q];
  }
  __syncthreads();
  // H = J^T W J, b = -J^T W e
  for (int idx = tid; idx < 34 * 34; idx += blockDim.x) {
    const int i = idx / 34, j = idx % 34;
    if (j < i) continue;
    double acc = 0.0;
    for (int k = 0; k < 18; ++k) acc += S.J[k * 34 + i] * S.WJ[k * 34 + j];
    S.H[i * 34 + j] = acc;
  }
  if (tid < 34) {
    double acc = 0.0;
    for (int k = 0; k < 18; ++k) acc += S.WJ[k * 34 + tid] * S.e[k];
    S.b[tid] = -acc;
  }
  if (tid == 64) {
    double ce = 0.0;
    for (int r = 0; r < 18; ++r) {
      double wr = 0.0;
      for (int k = 0; k < 18; ++k) wr += c->Wimu[r * 18 + k] * S.e[k];
      ce += S.e[r] * wr;
    }
    S.cost_imu = ce;
  }
  __syncthreads();
  // + pixel terms: ICP on x1 pose; photometric: H12 = B H6 B^T, b12 = B g6, B = [-M; I]
  for (int idx = tid; idx < 12 * 12; idx += blockDim.x) {
    const int i = idx / 12, j = idx % 12;
    if (j < i) continue;
    const int a = i / 6, bb = j / 6, ii = i % 6, jj = j % 6;
    double v;
    if (a == 1 && bb == 1) {
      v = S.Hl[1][ii * 6 + jj];
    } else if (a == 0 && bb == 1) {      // -(M H6)_{ii jj}
      v = 0.0;
      for (int k = 0; k < 6; ++k) v -= S.M6[ii * 6 + k] * S.Hl[1][k * 6 + jj];
    } else {                              // (M H6 M^T)_{ii jj}
      v = 0.0;
      for (int k = 0; k < 6; ++k)
        for (int l = 0; l < 6; ++l) v += S.M6[ii * 6 + k] * S.Hl[1][k * 6 + l] * S.M6[jj * 6 + l];
    }
    const int gi = a == 0 ? ii : 17 + ii, gj = bb == 0 ? jj : 17 + jj;
    double add = v;
    if (a == 1 && bb == 1) add += S.Hl[0][ii * 6 + jj];
    S.H[gi * 34 + gj] += add;
  }
  if (tid < 6) {
    double g0 = 0.0;
    for (int k = 0; k < 6; ++k) g0 -= S.M6[tid * 6 + k] * S.gl[1][k];
    S.b[tid] += g0;
    S.b[17 + tid] += S.gl[1][tid] + S.gl[0][tid];
  }
  __syncthreads();
  // + prior on x0: H00 += H*, b0 += b* - H* (x0 boxminus xbar)
  __shared__ double s_dprior[17];
  if (tid == 0) state_boxminus(c->x0, c->xbar, s_dprior);
  __syncthreads();
  for (int idx = tid; idx < 17 * 17; idx += blockDim.x) {
    const int i = idx / 17, j = idx % 17;
    if (j >= i) S.H[i * 34 + j] += c->Hs[i * 17 + j];
  }
  if (tid < 17) {
    double acc = c->bs[tid];
    for (int k = 0; k < 17; ++k) acc -= c->Hs[tid * 17 + k] * s_dprior[k];
    S.b[tid] += acc;
  }
  __syncthreads();
  // mirror the upper triangle
  for (int idx = tid; idx < 34 * 34; idx += blockDim.x) {
    const int i = idx / 34, j = idx % 34;
    if (j < i) S.H[i * 34 + j] = S.H[j * 34 + i];
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kSolveThreads) k_gn_step(SolveParams sp) {
  Ctrl* c = sp.ctrl;
  if (c->status != 0) return;
  __shared__ StepShared S;
  __shared__ double A[34 * 34];
  __shared__ double x[34];
  assemble(sp, S);
  const int tid = threadIdx.x;
  if (!S.ok) {
    if (tid == 0) c->status = DRI_ENOTREADY;
    return;
  }
  // Jacobi-scaled Cholesky solve of H dx = b
  if (tid < 34) S.scale[tid] = 1.0 / sqrt(fmax(S.H[tid * 34 + tid], 1e-300));
  __syncthreads();
  for (int idx = tid; idx < 34 * 34; idx += blockDim.x) {
    const int i = idx / 34, j = idx % 34;
    A[idx] = S.H[idx] * S.scale[i] * S.scale[j];
  }
  if (tid < 34) x[tid] = S.b[tid] * S.scale[tid];
  __syncthreads();
  const bool pd = block_cholesky(A, 34, 34);
  if (tid == 0) {
    bool good = pd;
    if (good) {
      chol_subst(A, 34, 34, x);
      for (int i = 0; i < 34; ++i) {
        x[i] *= S.scale[i];
        good = good && isfinite(x[i]);
      }
    }
    if (!good) {
      c->status = DRI_ELOST;
    } else {
      state_boxplus(c->x0, x);
      state_boxplus(c->x1, x + 17);
      const double* s = c->sums;
      c->n_icp[sp.level] = (int32_t)s[28];
      c->n_rgb[sp.level] = (int32_t)s[kSums + 28];
      c->cost = sp.W_icp * s[27] + sp.W_rgb * s[kSums + 27] + S.cost_imu;
      c->iterations += 1;
      write_transforms(c);
    }
  }
  __syncthreads();
  if (sp.last && c->status == 0) {
    for (int idx = tid; idx < 34 * 34; idx += blockDim.x) c->H[idx] = S.H[idx];
    if (tid < 34) {
      c->b[tid] = S.b[tid];
      c->d[tid] = x[tid];
    }
  }
}

__device__ void load_pose_ref(Ctrl* c) {
  quat_to_rot(c->x.q, c->Rref);
  for (int i = 0; i < 3; ++i) c->rref[i] = c->x.r[i];
}

// W_IMU at c->x0 (noise propagated through the recursion, Sigma^-1), and the
// IMU prediction x^1(x0).  Whole block; returns false (status set) on failure.
__device__ bool imu_weight_and_prediction(const SolveParams& sp, Ctrl* c, DState* x1_pred) {
  const int tid = threadIdx.x;
  __shared__ Preint P;
  __shared__ Pred pr;
  __shared__ int s_np, s_ok;
  __shared__ int pk[kMaxPieces];
  __shared__ double pdt[kMaxPieces];
  __shared__ double G[81], GS[81], L[81], Winv[81];
  if (tid == 0) {
    s_ok = 1;
    if (!c->initialised || fabs(sp.imu->t0 - c->t_state) > 1e-9) s_ok = 0;
    s_np = s_ok ? imu_pieces(sp.imu, pk, pdt) : -1;
    if (s_np <= 0) s_ok = 0;
    if (s_ok) {
      preintegrate(sp.imu, pk, pdt, s_np, c->x0.bg, c->x0.ba, true, sp.gyr_nd, sp.acc_nd, P);
      predict(c->x0, P, sp, pr);
      // G = d(r^, a^, v^) / d(dphi, dv, dp)
      for (int i = 0; i < 81; ++i) G[i] = 0.0;
      double Rrc[3], K[9], KR[9], QA[9];
      m3_vec(pr.R, sp.r_CS, Rrc);
      hat3(Rrc, K);
      m3_mul(K, pr.RWS1, KR);
      m3_mul(pr.Q0, pr.A0, QA);
      for (int r = 0; r < 3; ++r)
        for (int q = 0; q < 3; ++q) {
          G[r * 9 + q] = KR[r * 3 + q];
          G[r * 9 + 6 + q] = pr.A0[r * 3 + q];
          G[(3 + r) * 9 + q] = pr.RWS1[r * 3 + q];
          G[(6 + r) * 9 + 3 + q] = QA[r * 3 + q];
        }
    } else {
      c->status = DRI_ENOTREADY;
    }
  }
  __syncthreads();
  if (!s_ok) return false;
  // G Sigma_pre G^T, symmetrised
  if (tid < 81) {
    const int r = tid / 9, q = tid % 9;
    double acc = 0.0;
    for (int k = 0; k < 9; ++k) acc += G[r * 9 + k] * P.Sig[k * 9 + q];
    GS[tid] = acc;
  }
  __syncthreads();
  if (tid < 81) {
    const int r = tid / 9, q = tid % 9;
    double acc = 0.0;
    for (int k = 0; k < 9; ++k) acc += GS[r * 9 + k] * G[q * 9 + k];
    L[tid] = acc;
  }
  __syncthreads();
  double sym = 0.0;
  if (tid < 81) sym = 0.5 * (L[tid] + L[(tid % 9) * 9 + tid / 9]);
  __syncthreads();
  if (tid < 81) L[tid] = sym;
  __syncthreads();
  const bool pd = block_cholesky(L, 9, 9);
  if (tid < 9) {
    double col[9];
    for (int i = 0; i < 9; ++i) col[i] = (i == tid) ? 1.0 : 0.0;
    chol_subst(L, 9, 9, col);
    for (int i = 0; i < 9; ++i) Winv[i * 9 + tid] = col[i];
  }
  __syncthreads();
  for (int idx = tid; idx < 18 * 18; idx += blockDim.x) {
    const int r = idx / 18, q = idx % 18;
    double w = 0.0;
    if (r < 9 && q < 9) {
      w = 0.5 * (Winv[r * 9 + q] + Winv[q * 9 + r]);
    } else if (r == q) {
      if (r < 12) w = 1.0 / (sp.gyr_rw * sp.gyr_rw * P.T);
      else if (r < 15) w = 1.0 / (sp.acc_rw * sp.acc_rw * P.T);
      else w = 1.0 / (sp.sigma_grav * sp.sigma_grav);
    }
    c->Wimu[idx] = w;
  }
  if (tid == 0) {
    if (!pd) c->status = DRI_ELOST;
    if (x1_pred) {
      // x1 := x^1(x0): biases and q_IW carried over
      DState x1 = c->x0;
      for (int i = 0; i < 3; ++i) {
        x1.r[i] = pr.r[i];
        x1.v[i] = pr.v[i];
      }
      rot_to_quat(pr.R, x1.q);
      *x1_pred = x1;
    }
  }
  __syncthreads();
  return pd;
}

__global__ void __launch_bounds__(kSolveThreads) k_frame_begin(SolveParams sp) {
  Ctrl* c = sp.ctrl;
  const int tid = threadIdx.x;
  if (tid == 0) {
    c->status = 0;
    c->xstart = c->x;
    c->x0 = c->x;
    c->iterations = 0;
    c->cost = 0.0;
    for (int l = 0; l < kMaxLevels; ++l) c->n_icp[l] = c->n_rgb[l] = 0;
  }
  __syncthreads();
  if (imu_weight_and_prediction(sp, c, &c->x1) && tid == 0) write_transforms(c);
}

__global__ void __launch_bounds__(kSolveThreads) k_frame_end(SolveParams sp) {
  Ctrl* c = sp.ctrl;
  const int tid = threadIdx.x;
  __shared__ int s_ok;
  if (tid == 0) {
    if (c->status == 0 && c->n_icp[0] + c->n_rgb[0] < sp.min_valid) c->status = DRI_ELOST;
    s_ok = c->status == 0;
  }
  __syncthreads();
  if (!s_ok) {
    if (tid == 0) c->x = c->xstart;
    return;
  }
  // b' = b - H d; Schur complement of the x0 block (Eq. 8)
  __shared__ double H[34 * 34];
  __shared__ double bp[34];
  __shared__ double L[17 * 17];
  __shared__ double X[17 * 18];
  for (int idx = tid; idx < 34 * 34; idx += blockDim.x) H[idx] = c->H[idx];
  __syncthreads();
  if (tid < 34) {
    double acc = c->b[tid];
    for (int k = 0; k < 34; ++k) acc -= H[tid * 34 + k] * c->d[k];
    bp[tid] = acc;
  }
  for (int idx = tid; idx < 17 * 17; idx += blockDim.x) L[idx] = H[(idx / 17) * 34 + idx % 17];
  __syncthreads();
  const bool pd = block_cholesky(L, 17, 17);
  if (tid < 18) {
    double col[17];
    for (int i = 0; i < 17; ++i) col[i] = tid < 17 ? H[i * 34 + 17 + tid] : bp[i];
    chol_subst(L, 17, 17, col);
    for (int i = 0; i < 17; ++i) X[i * 18 + tid] = col[i];
  }
  __syncthreads();
  __shared__ double Hs[17 * 17], bs[17];
  for (int idx = tid; idx < 17 * 17; idx += blockDim.x) {
    const int i = idx / 17, j = idx % 17;
    double acc = H[(17 + i) * 34 + 17 + j];
    for (int k = 0; k < 17; ++k) acc -= H[(17 + i) * 34 + k] * X[k * 18 + j];
    Hs[idx] = acc;
  }
  if (tid < 17) {
    double acc = bp[17 + tid];
    for (int k = 0; k < 17; ++k) acc -= H[(17 + tid) * 34 + k] * X[k * 18 + 17];
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
  for (int idx = tid; idx < 17 * 17; idx += blockDim.x) {
    const int i = idx / 17, j = idx % 17;
    c->Hs[idx] = 0.5 * (Hs[i * 17 + j] + Hs[j * 17 + i]);
  }
  if (tid < 17) c->bs[tid] = bs[tid];
  if (tid == 0) {
    c->x = c->x1;
    c->xbar = c->x1;
    c->t_state = sp.imu->t1;
    load_pose_ref(c);
    c->ref_index = 1 - c->ref_index;
  }
}

__global__ void k_frame_init(SolveParams sp) {
  const double t_frame = sp.imu->t1;
  Ctrl* c = sp.ctrl;
  const int tid = threadIdx.x;
  if (tid < 17 * 17) {
    const int i = tid / 17, j = tid % 17;
    double v = 0.0;
    if (i == j) {
      const double s = i < 6 ? sp.prior_sigma[0]
                     : i < 9 ? sp.prior_sigma[1]
                     : i < 12 ? sp.prior_sigma[2]
                     : i < 15 ? sp.prior_sigma[3] : sp.prior_sigma[4];
      v = 1.0 / (s * s);
    }
    c->Hs[tid] = v;
  }
  if (tid < 17) c->bs[tid] = 0.0;
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
    for (int l = 0; l < kMaxLevels; ++l) c->n_icp[l] = c->n_rgb[l] = 0;
  }
}

__global__ void __launch_bounds__(kSolveThreads) k_linearise_begin(SolveParams sp, DState x0, DState x1) {
  Ctrl* c = sp.ctrl;
  const int tid = threadIdx.x;
  if (tid == 0) {
    c->status = 0;
    c->x0 = x0;
    c->x1 = x1;
  }
  __syncthreads();
  if (imu_weight_and_prediction(sp, c, nullptr) && tid == 0) write_transforms(c);
}

__global__ void __launch_bounds__(kSolveThreads) k_linearise_end(SolveParams sp, dri_linearisation* out) {
  Ctrl* c = sp.ctrl;
  __shared__ StepShared S;
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
  if (tid < 18) out->e_imu[tid] = S.ok ? S.e[tid] : 0.0;
  if (tid == 0) {
    const double* s = c->sums;
    out->cost_icp = sp.W_icp * s[27];
    out->cost_rgb = sp.W_rgb * s[kSums + 27];
    out->cost_imu = S.ok ? S.cost_imu : 0.0;
    out->n_icp = (int64_t)s[28];
    out->n_rgb = (int64_t)s[kSums + 28];
    if (!S.ok) c->status = DRI_ENOTREADY;
  }
}

}  // namespace

cudaError_t launch_frame_begin(const SolveParams& p, cudaStream_t s) {
  k_frame_begin<<<1, kSolveThreads, 0, s>>>(p);
  return cudaGetLastError();
}
cudaError_t launch_gn_step(const SolveParams& p, cudaStream_t s) {
  k_gn_step<<<1, kSolveThreads, 0, s>>>(p);
  return cudaGetLastError();
}
cudaError_t launch_frame_end(const SolveParams& p, cudaStream_t s) {
  k_frame_end<<<1, kSolveThreads, 0, s>>>(p);
  return cudaGetLastError();
}
cudaError_t launch_frame_init(const SolveParams& p, cudaStream_t s) {
  k_frame_init<<<1, 320, 0, s>>>(p);
  return cudaGetLastError();
}
cudaError_t launch_linearise_begin(const SolveParams& p, const DState& x0, const DState& x1,
                                   cudaStream_t s) {
  k_linearise_begin<<<1, kSolveThreads, 0, s>>>(p, x0, x1);
  return cudaGetLastError();
}
cudaError_t launch_linearise_end(const SolveParams& p, dri_linearisation* out, cudaStream_t s) {
  k_linearise_end<<<1, kSolveThreads, 0, s>>>(p, out);
  return cudaGetLastError();
}

}  // namespace dri
