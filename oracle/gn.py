"""Joint cost, Gauss-Newton, marginalisation and the per-frame tracker.

Oracle code (test infrastructure only).

Cost (Eq. 6): photometric + ICP + IMU terms and the marginalisation prior
  (x_0 boxminus xbar_0 - H*^-1 b*)^T H* (x_0 boxminus xbar_0 - H*^-1 b*).
System (Eq. 7): H dx = b over dx = [dx_0; dx_1] (34-D), H = sum J^T W J,
b = -sum J^T W e; solved by dense Cholesky; both states updated with boxplus
after each iteration (Sec. IV-D), coarse-to-fine over the pyramid levels.

Prior (reading of Eq. 9, whose Delta x is not defined): the prior adds H* to
H_00 and b* - H* (x_0 boxminus xbar_0) to b_0.  This is the gradient of Eq. 6's
prior term (its Jacobian taken as the identity) and equals Eq. 9b with
Delta x := xbar_0 boxminus x_0.

Marginalisation (Eq. 8): after the last update the last system is moved to the
new point to first order (b <- b - H dx_last) and x_0 is removed with the Schur
complement H* = H_11 - H_10 H_00^-1 H_01, b* = b_1 - H_10 H_00^-1 b_0; xbar := x_1.

IMU term per iteration: re-integrated at x_0's biases (imu_mode 0), or the
first-order bias update of the pre-integration made at the frame's
linearisation point, which moves to x_0's current biases (with a
re-integration) once they leave the thresholds (imu_mode 1, params.py).

RGB-D-only baseline (track_mode 1, params.py): Gauss-Newton on x_1's pose
alone with H_icp + lambda H_rgb, x_0 fixed, no IMU term, prior or
marginalisation (`track_pose_only`).

Gyro-only variant (track_mode 2, params.py): the joint system with the IMU
term's accelerometer-related rows at zero weight (`imu.weight_gyro_only`) and
the velocity, accelerometer bias and gravity of both states held (`hold`);
x_1 starts at x_0's position with the gyro's rotation prediction; the prior
keeps no information on the held components.

Frame loop (reading; the paper does not state the initialisation): x_0 := the
previous x_1, x_1 := the IMU prediction x^_1(x_0); W_IMU computed there.  The
first frame only initialises: x_1 := x_init (identity pose, W = first camera
frame, Sec. II), the diagonal first-frame prior, and the frame becomes the
reference.  After every tracked frame the live frame's maps become the next
reference at the final T_WC1.
"""
from __future__ import annotations

import numpy as np

from . import imu as imu_mod
from .maps import frame_levels, reference_from_frame
from .photogeo import linearise
from .so3 import State, boxminus, boxplus

POSE0 = slice(0, 6)
POSE1 = slice(17, 23)
HELD_GYRO_ONLY = np.r_[6:9, 12:17]      # v, b_a, gravity of one state (track_mode 2)


def first_prior(cfg):
    s = cfg.prior_sigma
    sig = np.concatenate([[s["pose"]] * 6, [s["v"]] * 3, [s["bg"]] * 3, [s["ba"]] * 3,
                          [s["grav"]] * 2])
    return np.diag(1.0 / sig ** 2), np.zeros(17)


def prior_terms(x0, xbar, Hs, bs):
    """Contribution of the prior to (H_00, b_0)."""
    d = boxminus(x0, xbar)
    return Hs, bs - Hs @ d


def prior_cost(x0, xbar, Hs, bs):
    d = boxminus(x0, xbar) - np.linalg.solve(Hs, bs)
    return float(d @ Hs @ d)


def assemble(lin, J_imu, e_imu, W_imu, x0, xbar, Hs, bs):
    """The 34 x 34 Gauss-Newton system of Eq. 7."""
    H = np.zeros((34, 34))
    b = np.zeros(34)
    idx = np.r_[0:6, 17:23]
    H[np.ix_(idx, idx)] += lin["H_rgb"]
    b[idx] += lin["b_rgb"]
    H[POSE1, POSE1] += lin["H_icp"]
    b[POSE1] += lin["b_icp"]
    H += J_imu.T @ W_imu @ J_imu
    b += -J_imu.T @ W_imu @ e_imu
    Hp, bp = prior_terms(x0, xbar, Hs, bs)
    H[0:17, 0:17] += Hp
    b[0:17] += bp
    return H, b


def hold(H, b, dims):
    """Removes the tangent components `dims` from the system H dx = b (in
    place): their rows and columns become the identity's and their right-hand
    side zero, so their step is exactly zero and the other components solve
    the system without them."""
    H[dims, :] = 0.0
    H[:, dims] = 0.0
    H[dims, dims] = 1.0
    b[dims] = 0.0


def cholesky_solve(H, b):
    L = np.linalg.cholesky(H)
    y = np.linalg.solve(L, b)
    return np.linalg.solve(L.T, y)


def schur(H, b):
    """Eq. 8: marginalise the first 17 coordinates."""
    H00, H01, H10, H11 = H[:17, :17], H[:17, 17:], H[17:, :17], H[17:, 17:]
    X = np.linalg.solve(H00, np.column_stack([H01, b[:17]]))
    return H11 - H10 @ X[:, :17], b[17:] - H10 @ X[:, 17]


class TrackingLost(RuntimeError):
    pass


class Tracker:
    """Per-stream FP64 tracker: the oracle of one dri_track call per frame."""

    def __init__(self, cfg, x_init, t_init=None):
        self.cfg = cfg
        self.x = State.from_dict(x_init) if isinstance(x_init, dict) else x_init.copy()
        self.t = t_init
        self.ref = None
        self.T_ref = None
        self.Hs, self.bs = first_prior(cfg)
        self.xbar = self.x.copy()
        self.imu = np.zeros((0, 7))
        self.lin = None             # imu_mode 1: (pre-integration, b_g, b_a) of the frame

    def preintegration(self, x0, t0, t1):
        """The pre-integration the current iteration uses (module docstring)."""
        cfg = self.cfg
        if cfg.imu_mode != 1 or self.lin is None:
            return imu_mod.preintegrate(self.imu, t0, t1, x0.bg, x0.ba)
        pre, bg, ba = self.lin
        dbg, dba = x0.bg - bg, x0.ba - ba
        if np.linalg.norm(dbg) > cfg.bias_relin_g or np.linalg.norm(dba) > cfg.bias_relin_a:
            pre = imu_mod.preintegrate(self.imu, t0, t1, x0.bg, x0.ba)
            self.lin = (pre, x0.bg.copy(), x0.ba.copy())
            return pre
        return imu_mod.correct(pre, dbg, dba)

    def first_iterate(self, x0, pre):
        """x_1's starting point: the IMU prediction x^_1(x_0) with x_0's biases
        and gravity; in the gyro-only variant x_0's position and velocity with
        the predicted rotation R_WC0 R_CS dR R_CS^T."""
        from .so3 import rot_to_quat
        pr = imu_mod.predict(x0, pre, self.cfg)
        q = rot_to_quat(pr["R"])
        if self.cfg.track_mode == 2:
            return State(x0.r.copy(), q, x0.v.copy(), x0.bg.copy(), x0.ba.copy(), x0.qg.copy())
        return State(pr["r"], q, pr["v"], x0.bg.copy(), x0.ba.copy(), x0.qg.copy())

    def set_reference(self, ref, R_ref, r_ref):
        """Replaces the reference with uploaded levels (maps.reference_from_upload)."""
        self.ref = ref
        self.T_ref = (np.asarray(R_ref, dtype=np.float64), np.asarray(r_ref, dtype=np.float64).copy())

    def push_imu(self, samples):
        self.imu = np.concatenate([self.imu, np.asarray(samples, dtype=np.float64)])

    def linearise_all(self, levels, l, x0, x1, t0, t1, W_imu):
        """All terms of Eq. 6 at (x0, x1) on level l: returns (H, b, parts)."""
        cfg = self.cfg
        lin = linearise(levels[l], self.ref[l], self.T_ref[0], self.T_ref[1], x0, x1, cfg)
        pre = self.preintegration(x0, t0, t1)
        e, pr = imu_mod.residual(x0, x1, pre, cfg)
        J = imu_mod.jacobian(x0, x1, pre, cfg, e, pr)
        H, b = assemble(lin, J, e, W_imu, x0, self.xbar, self.Hs, self.bs)
        if cfg.track_mode == 2:
            hold(H, b, np.r_[HELD_GYRO_ONLY, 17 + HELD_GYRO_ONLY])
        parts = dict(lin=lin, e_imu=e, J_imu=J, cost_imu=float(e @ W_imu @ e))
        return H, b, parts

    def track(self, depth, intensity, t):
        cfg = self.cfg
        levels = frame_levels(depth, intensity, cfg)
        if self.ref is None:                       # first frame: initialise only
            self.t = t
            self.T_ref = (self.x.R, self.x.r.copy())
            self.ref = reference_from_frame(levels, *self.T_ref, fp16=self.cfg.fp16_maps)
            self.xbar = self.x.copy()
            return dict(status="init", x1=self.x.copy())
        if cfg.track_mode == 1:
            return self.track_pose_only(levels, t)
        t0, t1 = self.t, t
        x0 = self.x.copy()
        W_imu, S_imu = imu_mod.weight(x0, self.imu, t0, t1, cfg)
        pre = imu_mod.preintegrate(self.imu, t0, t1, x0.bg, x0.ba)
        self.lin = (pre, x0.bg.copy(), x0.ba.copy())
        if cfg.track_mode == 2:
            W_imu = imu_mod.weight_gyro_only(S_imu)
        x1 = self.first_iterate(x0, pre)
        counts = {}
        points = {}                              # per level: the last (x0, x1) linearised at
        H = b = d = None
        for l in range(cfg.levels - 1, -1, -1):
            for _ in range(cfg.iters[l]):
                points[l] = (x0.copy(), x1.copy())
                H, b, parts = self.linearise_all(levels, l, x0, x1, t0, t1, W_imu)
                counts[l] = (parts["lin"]["n_icp"], parts["lin"]["n_rgb"])
                try:
                    d = cholesky_solve(H, b)
                except np.linalg.LinAlgError as exc:
                    raise TrackingLost("Cholesky failed") from exc
                if not np.all(np.isfinite(d)):
                    raise TrackingLost("non-finite step")
                x0 = boxplus(x0, d[:17])
                x1 = boxplus(x1, d[17:])
        if counts[0][0] + counts[0][1] < cfg.min_valid:
            raise TrackingLost("too few correspondences")
        Hs, bs = schur(H, b - H @ d)
        if cfg.track_mode == 2:                # no information on the held components
            Hs[HELD_GYRO_ONLY, :] = 0.0
            Hs[:, HELD_GYRO_ONLY] = 0.0
            bs[HELD_GYRO_ONLY] = 0.0
        self.Hs, self.bs = Hs, bs
        self.xbar = x1.copy()
        self.x = x1.copy()
        self.t = t1
        self.T_ref = (x1.R, x1.r.copy())
        self.ref = reference_from_frame(levels, *self.T_ref, fp16=self.cfg.fp16_maps)
        keep = np.searchsorted(self.imu[:, 0], t1, side="right") - 1
        self.imu = self.imu[max(keep, 0):]
        return dict(status="ok", x0=x0, x1=x1, counts=counts, points=points, H=H, b=b, d_last=d,
                    H_prior=Hs, b_prior=bs)

    def track_pose_only(self, levels, t):
        """RGB-D-only baseline (track_mode 1, params.py): Gauss-Newton on x_1's
        pose with H = H_icp + lambda H_rgb(x_1 block), x_0 fixed."""
        cfg = self.cfg
        x0 = self.x.copy()
        x1 = self.x.copy()
        lam = cfg.rgbd_lambda
        counts = {}
        H = b = None
        for l in range(cfg.levels - 1, -1, -1):
            for _ in range(cfg.iters[l]):
                lin = linearise(levels[l], self.ref[l], self.T_ref[0], self.T_ref[1], x0, x1, cfg)
                counts[l] = (lin["n_icp"], lin["n_rgb"])
                H = lin["H_icp"] + lam * lin["H_rgb"][6:, 6:]
                b = lin["b_icp"] + lam * lin["b_rgb"][6:]
                try:
                    d = cholesky_solve(H, b)
                except np.linalg.LinAlgError as exc:
                    raise TrackingLost("Cholesky failed") from exc
                if not np.all(np.isfinite(d)):
                    raise TrackingLost("non-finite step")
                x1 = boxplus(x1, np.concatenate([d, np.zeros(11)]))
        if counts[0][0] + counts[0][1] < cfg.min_valid:
            raise TrackingLost("too few correspondences")
        self.x = x1.copy()
        self.xbar = x1.copy()
        self.t = t
        self.T_ref = (x1.R, x1.r.copy())
        self.ref = reference_from_frame(levels, *self.T_ref, fp16=self.cfg.fp16_maps)
        return dict(status="ok", x0=x0, x1=x1, counts=counts, H=H, b=b)
