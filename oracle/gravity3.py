"""The 3-D gravity-with-gauge form of the state (Sec. II and IV-A).

Oracle code (test infrastructure only).  The CUDA path solves the 2-DoF form
(so3.py); this module is the paper's own parameterisation, for comparison.

The paper keeps q_IW with three degrees of freedom although two fix the
direction of gravity.  Here the gravity perturbation is dg in R^3,
q_IW <- exp(dg) (x) q_IW, so a state's tangent space has 18 dimensions
(dr, da, dv, dbg, dba, dg) and the joint system 36.  Turning the inertial
frame about gravity (I's z) together with v_I changes no measurement
(tests/test_oracle_imu_gauge.py): that direction is the gauge freedom.  Only
the priors see it -- the first-frame prior, here on all three gravity axes,
and what marginalisation carries forward through the gravity random walk --
so the system stays regular but is weak along it.  Readings (the paper gives
no damping): each Gauss-Newton step is damped as Levenberg-Marquardt does on
the gravity blocks of both states, (H + mu D_g) dx = b with D_g the identity
on those 6 coordinates and mu = 1 (sigma 1 rad, weak against the first
prior's 0.1 rad); the damping regularises the step only and is not part of
the cost, so marginalisation takes the Schur complement of the undamped
system.  Everything else is the 2-DoF tracker's (gn.py): the pixel terms act
on the pose blocks, the IMU term is the same 18-D error with its 3 x 3 gravity
blocks kept whole (imu.gravity_blocks), x_1 starts at the IMU prediction, the
prior adds H* to H_00 and b* - H* (x_0 boxminus xbar) to b_0.
"""
from __future__ import annotations

import numpy as np

from . import gn
from . import imu as imu_mod
from .maps import frame_levels, reference_from_frame
from .photogeo import linearise
from .so3 import State, quat_conj, quat_exp, quat_log, quat_mul

DIM = 18
POSE0 = slice(0, 6)
POSE1 = slice(18, 24)
GRAV = np.r_[15:18, 33:36]          # gravity coordinates of x_0 and x_1 in the joint system


def boxplus(x, d):
    """x boxplus dx with dg in R^3: q_IW <- exp(dg) (x) q_IW; the rest as Eq. 2."""
    d = np.asarray(d, dtype=np.float64)
    q = quat_mul(quat_exp(d[3:6]), x.q)
    qg = quat_mul(quat_exp(d[15:18]), x.qg)
    return State(x.r + d[0:3], q / np.linalg.norm(q), x.v + d[6:9], x.bg + d[9:12],
                 x.ba + d[12:15], qg / np.linalg.norm(qg))


def boxminus(x, y):
    """x boxminus y with the whole rotation vector of q_IW,x (x) q_IW,y^-1."""
    out = np.zeros(DIM)
    out[0:3] = x.r - y.r
    out[3:6] = quat_log(quat_mul(x.q, quat_conj(y.q)))
    out[6:9] = x.v - y.v
    out[9:12] = x.bg - y.bg
    out[12:15] = x.ba - y.ba
    out[15:18] = quat_log(quat_mul(x.qg, quat_conj(y.qg)))
    return out


def imu_jacobian(x0, x1, pre, cfg, e=None, pr=None):
    """de_IMU / d(dx_0, dx_1), 18 x 36: the 2-DoF Jacobian's columns, with the
    gravity blocks of both states taken whole."""
    if e is None:
        e, pr = imu_mod.residual(x0, x1, pre, cfg)
    J2 = imu_mod.jacobian(x0, x1, pre, cfg, e, pr)
    G = imu_mod.gravity_blocks(x0, pre, cfg, e, pr)
    J = np.zeros((18, 2 * DIM))
    J[:, 0:15] = J2[:, 0:15]
    J[:, 18:33] = J2[:, 17:32]
    J[0:3, 15:18] = G["r0"]
    J[6:9, 15:18] = G["v0"]
    J[15:18, 15:18] = G["g0"]
    J[15:18, 33:36] = G["g1"]
    return J


def first_prior(cfg):
    """The first-frame prior of gn.first_prior with sigma_g on all three
    gravity axes."""
    s = cfg.prior_sigma
    sig = np.concatenate([[s["pose"]] * 6, [s["v"]] * 3, [s["bg"]] * 3, [s["ba"]] * 3,
                          [s["grav"]] * 3])
    return np.diag(1.0 / sig ** 2), np.zeros(DIM)


def assemble(lin, J_imu, e_imu, W_imu, x0, xbar, Hs, bs):
    """The undamped 36 x 36 system of Eq. 7."""
    H = np.zeros((2 * DIM, 2 * DIM))
    b = np.zeros(2 * DIM)
    idx = np.r_[0:6, 18:24]
    H[np.ix_(idx, idx)] += lin["H_rgb"]
    b[idx] += lin["b_rgb"]
    H[POSE1, POSE1] += lin["H_icp"]
    b[POSE1] += lin["b_icp"]
    H += J_imu.T @ W_imu @ J_imu
    b += -J_imu.T @ W_imu @ e_imu
    d = boxminus(x0, xbar)
    H[0:DIM, 0:DIM] += Hs
    b[0:DIM] += bs - Hs @ d
    return H, b


def schur(H, b):
    """Eq. 8 over x_0's 18 coordinates."""
    H00, H01, H10, H11 = H[:DIM, :DIM], H[:DIM, DIM:], H[DIM:, :DIM], H[DIM:, DIM:]
    X = np.linalg.solve(H00, np.column_stack([H01, b[:DIM]]))
    return H11 - H10 @ X[:, :DIM], b[DIM:] - H10 @ X[:, DIM]


class Tracker(gn.Tracker):
    """The per-frame tracker of gn.Tracker (RGB-D-inertial mode) with the 3-D
    gravity perturbation and the damped step."""

    def __init__(self, cfg, x_init, t_init=None, damping=1.0):
        if cfg.track_mode != 0:
            raise ValueError("the 3-D gravity form is built for the RGB-D-inertial tracker only")
        super().__init__(cfg, x_init, t_init)
        self.damping = float(damping)
        self.Hs, self.bs = first_prior(cfg)

    def linearise_all(self, levels, l, x0, x1, t0, t1, W_imu):
        cfg = self.cfg
        lin = linearise(levels[l], self.ref[l], self.T_ref[0], self.T_ref[1], x0, x1, cfg)
        pre = self.preintegration(x0, t0, t1)
        e, pr = imu_mod.residual(x0, x1, pre, cfg)
        J = imu_jacobian(x0, x1, pre, cfg, e, pr)
        H, b = assemble(lin, J, e, W_imu, x0, self.xbar, self.Hs, self.bs)
        return H, b, dict(lin=lin, e_imu=e, J_imu=J, cost_imu=float(e @ W_imu @ e))

    def step(self, H, b):
        """The damped Gauss-Newton step (H + mu D_g) dx = b."""
        Hd = H.copy()
        Hd[GRAV, GRAV] += self.damping
        return gn.cholesky_solve(Hd, b)

    def track(self, depth, intensity, t):
        cfg = self.cfg
        levels = frame_levels(depth, intensity, cfg)
        if self.ref is None:
            self.t = t
            self.T_ref = (self.x.R, self.x.r.copy())
            self.ref = reference_from_frame(levels, *self.T_ref, fp16=cfg.fp16_maps)
            self.xbar = self.x.copy()
            return dict(status="init", x1=self.x.copy())
        t0, t1 = self.t, t
        x0 = self.x.copy()
        W_imu, _ = imu_mod.weight(x0, self.imu, t0, t1, cfg)
        pre = imu_mod.preintegrate(self.imu, t0, t1, x0.bg, x0.ba)
        self.lin = (pre, x0.bg.copy(), x0.ba.copy())
        x1 = self.first_iterate(x0, pre)
        counts = {}
        H = b = d = None
        for l in range(cfg.levels - 1, -1, -1):
            for _ in range(cfg.iters[l]):
                H, b, parts = self.linearise_all(levels, l, x0, x1, t0, t1, W_imu)
                counts[l] = (parts["lin"]["n_icp"], parts["lin"]["n_rgb"])
                try:
                    d = self.step(H, b)
                except np.linalg.LinAlgError as exc:
                    raise gn.TrackingLost("Cholesky failed") from exc
                if not np.all(np.isfinite(d)):
                    raise gn.TrackingLost("non-finite step")
                x0 = boxplus(x0, d[:DIM])
                x1 = boxplus(x1, d[DIM:])
        if counts[0][0] + counts[0][1] < cfg.min_valid:
            raise gn.TrackingLost("too few correspondences")
        Hs, bs = schur(H, b - H @ d)
        self.Hs, self.bs = Hs, bs
        self.xbar = x1.copy()
        self.x = x1.copy()
        self.t = t1
        self.T_ref = (x1.R, x1.r.copy())
        self.ref = reference_from_frame(levels, *self.T_ref, fp16=cfg.fp16_maps)
        keep = np.searchsorted(self.imu[:, 0], t1, side="right") - 1
        self.imu = self.imu[max(keep, 0):]
        return dict(status="ok", x0=x0, x1=x1, counts=counts, H=H, b=b, d_last=d,
                    H_prior=Hs, b_prior=bs)
