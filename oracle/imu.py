"""Inertial pre-integration and the IMU error term (Sec. IV-C, Eq. 5).

Oracle code (test infrastructure only).  The paper integrates the IMU
"numerically between the previous and current camera frames" with the
pre-integration of Forster et al. and the error e_IMU = x^_1(x_0) boxminus x_1
(Eq. 5).  Readings used here:

Integration (zero-order hold).  Sample k at t_k holds on [t_k, t_{k+1}).  The
interval [t0, t1] is cut at every sample time inside it; the first piece uses
the last sample with t_k <= t0.  Per piece (dt, w = gyr - b_g, a = acc - b_a),
in this order:
  dp <- dp + dv dt + 1/2 dR a dt^2
  dv <- dv + dR a dt
  dR <- dR Exp(w dt)
By default the integration is repeated at x_0's current biases at every
Gauss-Newton iteration (exact).  Alongside it run the exact derivatives of this
recursion w.r.t. the biases (right perturbation of dR): Phi_g = d(dR)/d(b_g),
V_g, P_g = d(dv, dp)/d(b_g), V_a, P_a = d(dv, dp)/d(b_a).  `correct` is the
alternative of Forster et al. the paper builds on: a first-order update of a
pre-integration to new biases without re-integrating.

Prediction x^_1(x_0), with R_IS = R_IW R_WC R_CS, r_IS = R_IW (r_WC + R_WC r_CS),
g_I = (0, 0, -g), T = t1 - t0:
  R^_IS1 = R_IS0 dR,  v^_1 = v_0 + g_I T + R_IS0 dv,
  r^_IS1 = r_IS0 + v_0 T + 1/2 g_I T^2 + R_IS0 dp,
biases and q_IW carried over, then converted back to (r_WC, q_WC) with q_IW0.
Error (18-D, order r, a, v, b_g, b_a, g): e = x^_1 boxminus x_1 with full 3-D
logs for both orientations.

Weight.  W_IMU = Sigma^-1, Sigma block diagonal: the (r, a, v) block is
G Sigma_pre G^T with Sigma_pre the discrete propagation of the gyro and
accelerometer white noise through the recursion (per-piece covariance
density^2 / dt, Table I densities) and G the derivative of the prediction
w.r.t. the pre-integrated (dphi, dv, dp); the bias blocks are the random walks
density^2 T (Table I); the gravity block sigma_grav^2 I.  It is computed once
per frame, at the initial linearisation point.
"""
from __future__ import annotations

import numpy as np

from .so3 import exp_so3, hat, jl_inv, jr, jr_inv, log_so3

P2 = np.array([[1.0, 0.0], [0.0, 1.0], [0.0, 0.0]])   # gravity perturbation axes


class CoverageError(ValueError):
    pass


def pieces(samples, t0, t1):
    """Zero-order-hold pieces of [t0, t1] as (sample index, duration)."""
    ts = samples[:, 0]
    if len(ts) == 0 or ts[0] > t0 or ts[-1] < t1:
        raise CoverageError("IMU samples do not cover [t0, t1]")
    k = int(np.searchsorted(ts, t0, side="right") - 1)
    out = []
    tau = t0
    while tau < t1:
        nxt = t1 if k + 1 >= len(ts) else min(ts[k + 1], t1)
        if nxt > tau:
            out.append((k, nxt - tau))
        tau = nxt
        k += 1
    return out


def preintegrate(samples, t0, t1, bg, ba, gyr_nd=None, acc_nd=None):
    dR = np.eye(3)
    dv = np.zeros(3)
    dp = np.zeros(3)
    Phi_g = np.zeros((3, 3))
    V_g = np.zeros((3, 3))
    P_g = np.zeros((3, 3))
    V_a = np.zeros((3, 3))
    P_a = np.zeros((3, 3))
    cov = gyr_nd is not None
    Sig = np.zeros((9, 9))
    for k, dt in pieces(samples, t0, t1):
        w = samples[k, 1:4] - bg
        a = samples[k, 4:7] - ba
        th = w * dt
        E = exp_so3(th)
        Jr = jr(th)
        Ah = dR @ hat(a)
        P_g = P_g + V_g * dt - 0.5 * Ah @ Phi_g * dt * dt
        P_a = P_a + V_a * dt - 0.5 * dR * dt * dt
        V_g = V_g - Ah @ Phi_g * dt
        V_a = V_a - dR * dt
        Phi_g = E.T @ Phi_g - Jr * dt
        if cov:
            A = np.eye(9)
            A[0:3, 0:3] = E.T
            A[3:6, 0:3] = -Ah * dt
            A[6:9, 0:3] = -0.5 * Ah * dt * dt
            A[6:9, 3:6] = np.eye(3) * dt
            Bg = np.zeros((9, 3))
            Bg[0:3] = Jr * dt
            Ba = np.zeros((9, 3))
            Ba[3:6] = dR * dt
            Ba[6:9] = 0.5 * dR * dt * dt
            Sig = A @ Sig @ A.T + (gyr_nd ** 2 / dt) * Bg @ Bg.T + (acc_nd ** 2 / dt) * Ba @ Ba.T
        dp = dp + dv * dt + 0.5 * dR @ a * dt * dt
        dv = dv + dR @ a * dt
        dR = dR @ E
    return dict(dR=dR, dv=dv, dp=dp, Phi_g=Phi_g, V_g=V_g, P_g=P_g, V_a=V_a, P_a=P_a,
                Sigma=Sig, T=t1 - t0)


def correct(pre, dbg, dba):
    """First-order update of a pre-integration made at biases (b_g, b_a) to
    (b_g + dbg, b_a + dba), without re-integrating (Forster et al.):
      dR <- dR Exp(Phi_g dbg),  dv <- dv + V_g dbg + V_a dba,
      dp <- dp + P_g dbg + P_a dba.
    The update is linear in the biases except for the rotation, whose bias
    Jacobian at the new point is Jr(Phi_g dbg) Phi_g (derivative of
    Exp(Phi_g (dbg + e)) = Exp(Phi_g dbg) Exp(Jr(Phi_g dbg) Phi_g e) to first
    order in e); the others are unchanged, so the residual's Jacobian stays the
    exact derivative of the updated model."""
    dbg = np.asarray(dbg, dtype=np.float64)
    dba = np.asarray(dba, dtype=np.float64)
    th = pre["Phi_g"] @ dbg
    out = dict(pre)
    out["dR"] = pre["dR"] @ exp_so3(th)
    out["dv"] = pre["dv"] + pre["V_g"] @ dbg + pre["V_a"] @ dba
    out["dp"] = pre["dp"] + pre["P_g"] @ dbg + pre["P_a"] @ dba
    out["Phi_g"] = jr(th) @ pre["Phi_g"]
    return out


def predict(x0, pre, cfg):
    """x^_1(x_0): (r^_WC1, R^_WC1, v^_1) plus the intermediates the Jacobian uses."""
    R0, Q0, Rc, rc = x0.R, x0.Rg, cfg.R_CS, cfg.r_CS
    g_I = np.array([0.0, 0.0, -cfg.g])
    T = pre["T"]
    R_WS1 = R0 @ Rc @ pre["dR"]
    R_hat = R_WS1 @ Rc.T
    c = x0.v * T + 0.5 * g_I * T * T
    r_hat = x0.r + R0 @ rc + Q0.T @ c + R0 @ Rc @ pre["dp"] - R_hat @ rc
    v_hat = x0.v + g_I * T + Q0 @ R0 @ Rc @ pre["dv"]
    return dict(r=r_hat, R=R_hat, v=v_hat, c=c, R_WS1=R_WS1)


def residual(x0, x1, pre, cfg):
    pr = predict(x0, pre, cfg)
    e = np.zeros(18)
    e[0:3] = pr["r"] - x1.r
    e[3:6] = log_so3(pr["R"] @ x1.R.T)
    e[6:9] = pr["v"] - x1.v
    e[9:12] = x0.bg - x1.bg
    e[12:15] = x0.ba - x1.ba
    e[15:18] = log_so3(x0.Rg @ x1.Rg.T)
    return e, pr


def gravity_blocks(x0, pre, cfg, e, pr):
    """The IMU error's derivatives by a rotation dg of q_IW about all three of
    I's axes (q_IW <- exp(dg) (x) q_IW): rows r and v by x_0's dg, rows g by
    x_0's and by x_1's (3 x 3 each).  The 2-DoF state keeps their x and y
    columns; the 3-D gravity variant (gravity3.py) all three."""
    Q0, A0 = x0.Rg, x0.R @ cfg.R_CS
    return dict(r0=Q0.T @ hat(pr["c"]), v0=-hat(Q0 @ A0 @ pre["dv"]), g0=jl_inv(e[15:18]),
                g1=-jr_inv(e[15:18]))


def jacobian(x0, x1, pre, cfg, e=None, pr=None):
    """Analytic de_IMU / d(dx_0, dx_1), 18 x 34 (columns: x_0 tangent then x_1's)."""
    if e is None:
        e, pr = residual(x0, x1, pre, cfg)
    R0, Q0, Rc, rc = x0.R, x0.Rg, cfg.R_CS, cfg.r_CS
    T = pre["T"]
    I3 = np.eye(3)
    R_WS1 = pr["R_WS1"]
    A0 = R0 @ Rc
    Jla = jl_inv(e[3:6])
    G = gravity_blocks(x0, pre, cfg, e, pr)
    J = np.zeros((18, 34))
    # x_1 (columns 17..33)
    J[0:3, 17:20] = -I3
    J[3:6, 20:23] = -jr_inv(e[3:6])
    J[6:9, 23:26] = -I3
    J[9:12, 26:29] = -I3
    J[12:15, 29:32] = -I3
    J[15:18, 32:34] = G["g1"] @ P2
    # x_0 (columns 0..16)
    J[0:3, 0:3] = I3
    J[0:3, 3:6] = -hat(pr["r"] - x0.r - Q0.T @ pr["c"])
    J[3:6, 3:6] = Jla
    J[6:9, 3:6] = -Q0 @ hat(A0 @ pre["dv"])
    J[0:3, 6:9] = Q0.T * T
    J[6:9, 6:9] = I3
    J[0:3, 9:12] = A0 @ pre["P_g"] + hat(pr["R"] @ rc) @ R_WS1 @ pre["Phi_g"]
    J[3:6, 9:12] = Jla @ R_WS1 @ pre["Phi_g"]
    J[6:9, 9:12] = Q0 @ A0 @ pre["V_g"]
    J[9:12, 9:12] = I3
    J[0:3, 12:15] = A0 @ pre["P_a"]
    J[6:9, 12:15] = Q0 @ A0 @ pre["V_a"]
    J[12:15, 12:15] = I3
    J[0:3, 15:17] = G["r0"] @ P2
    J[6:9, 15:17] = G["v0"] @ P2
    J[15:18, 15:17] = G["g0"] @ P2
    return J


def weight(x0, samples, t0, t1, cfg):
    """W_IMU = Sigma^-1 at x_0 (covariance propagated through the recursion)."""
    pre = preintegrate(samples, t0, t1, x0.bg, x0.ba, cfg.gyr_nd, cfg.acc_nd)
    pr = predict(x0, pre, cfg)
    Rc, rc = cfg.R_CS, cfg.r_CS
    G = np.zeros((9, 9))
    G[0:3, 0:3] = hat(pr["R"] @ rc) @ pr["R_WS1"]
    G[0:3, 6:9] = x0.R @ Rc
    G[3:6, 0:3] = pr["R_WS1"]
    G[6:9, 3:6] = x0.Rg @ x0.R @ Rc
    T = pre["T"]
    S = np.zeros((18, 18))
    S[0:9, 0:9] = G @ pre["Sigma"] @ G.T
    S[9:12, 9:12] = np.eye(3) * cfg.gyr_rw ** 2 * T
    S[12:15, 12:15] = np.eye(3) * cfg.acc_rw ** 2 * T
    S[15:18, 15:18] = np.eye(3) * cfg.sigma_grav_rw ** 2
    return np.linalg.inv(S), S


GYRO_ROWS = np.r_[3:6, 9:12]      # rotation and gyro-bias rows of e_IMU


def weight_gyro_only(S):
    """Weight of the gyro-only IMU term (track_mode 2, params.py) from the full
    covariance S of `weight`: the rotation and gyro-bias rows get the inverse
    of their own block of S (their marginal covariance), every
    accelerometer-related row zero weight."""
    W = np.zeros((18, 18))
    W[np.ix_(GYRO_ROWS, GYRO_ROWS)] = np.linalg.inv(S[np.ix_(GYRO_ROWS, GYRO_ROWS)])
    return W
