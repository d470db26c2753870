"""Rotations, quaternions and the state manifold (Sec. II, Sec. IV-A, Eq. 1-2).

Oracle code (test infrastructure only).  Hamilton quaternions stored
(w, x, y, z).  Orientation perturbations are global (left):
q boxplus da = exp(da) (x) q, and p boxminus q = log(p (x) q^-1) (Eq. 2).

Gravity direction (reading of Sec. IV-A): the paper uses q_IW with three
degrees of freedom and gauge freedom; here its perturbation is two-dimensional,
dg = (dg_x, dg_y) about I's x and y axes, q_IW boxplus dg = exp([dg_x, dg_y, 0])
(x) q_IW.  Rotation about gravity (I's z) is the unobservable gauge and is held
fixed.  The per-state tangent space therefore has 17 dimensions ordered
(dr, da, dv, dbg, dba, dg).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

TANGENT_DIM = 17
SMALL = 1e-3


def hat(w):
    w = np.asarray(w, dtype=np.float64)
    return np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])


def exp_so3(w):
    """Rodrigues' formula; Taylor series below 1e-3 rad."""
    w = np.asarray(w, dtype=np.float64)
    th2 = float(w @ w)
    th = np.sqrt(th2)
    K = hat(w)
    if th < SMALL:
        a = 1.0 - th2 / 6.0 + th2 * th2 / 120.0
        b = 0.5 - th2 / 24.0 + th2 * th2 / 720.0
    else:
        a = np.sin(th) / th
        b = (1.0 - np.cos(th)) / th2
    return np.eye(3) + a * K + b * (K @ K)


def quat_mul(p, q):
    """Hamilton product p (x) q."""
    pw, px, py, pz = p
    qw, qx, qy, qz = q
    return np.array([
        pw * qw - px * qx - py * qy - pz * qz,
        pw * qx + px * qw + py * qz - pz * qy,
        pw * qy - px * qz + py * qw + pz * qx,
        pw * qz + px * qy - py * qx + pz * qw,
    ])


def quat_conj(q):
    return np.array([q[0], -q[1], -q[2], -q[3]])


def quat_exp(w):
    """exp of a rotation vector as a unit quaternion."""
    w = np.asarray(w, dtype=np.float64)
    th = float(np.linalg.norm(w))
    if th < SMALL:
        th2 = th * th
        s = 0.5 - th2 / 48.0 + th2 * th2 / 3840.0        # sin(th/2)/th
        c = 1.0 - th2 / 8.0 + th2 * th2 / 384.0          # cos(th/2)
    else:
        s = np.sin(0.5 * th) / th
        c = np.cos(0.5 * th)
    return np.array([c, s * w[0], s * w[1], s * w[2]])


def quat_log(q):
    """Rotation vector of a unit quaternion (shortest rotation)."""
    q = np.asarray(q, dtype=np.float64)
    if q[0] < 0:
        q = -q
    v = q[1:]
    n = float(np.linalg.norm(v))
    if n < 1e-12:
        return 2.0 * v / q[0]
    return 2.0 * np.arctan2(n, q[0]) * v / n


def quat_to_rot(q):
    w, x, y, z = np.asarray(q, dtype=np.float64) / np.linalg.norm(q)
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def rot_to_quat(R):
    """Via the log of the rotation (axis-angle), so it needs no case split."""
    return quat_exp(log_so3(R))


def log_so3(R):
    """Rotation vector of a rotation matrix (angles below pi - 1e-6)."""
    R = np.asarray(R, dtype=np.float64)
    c = np.clip(0.5 * (np.trace(R) - 1.0), -1.0, 1.0)
    th = float(np.arccos(c))
    v = np.array([R[2, 1] - R[1, 2], R[0, 2] - R[2, 0], R[1, 0] - R[0, 1]])
    if th < SMALL:
        return 0.5 * (1.0 + th * th / 6.0 + 7.0 * th ** 4 / 360.0) * v
    return th / (2.0 * np.sin(th)) * v


def jr(w):
    """Right Jacobian of SO(3): Exp(w + d) ~= Exp(w) Exp(Jr(w) d)."""
    w = np.asarray(w, dtype=np.float64)
    th2 = float(w @ w)
    th = np.sqrt(th2)
    K = hat(w)
    if th < SMALL:
        a = 0.5 - th2 / 24.0 + th2 * th2 / 720.0
        b = 1.0 / 6.0 - th2 / 120.0 + th2 * th2 / 5040.0
    else:
        a = (1.0 - np.cos(th)) / th2
        b = (th - np.sin(th)) / (th2 * th)
    return np.eye(3) - a * K + b * (K @ K)


def jl_inv(w):
    """Inverse left Jacobian: Log(Exp(d) Exp(w)) ~= w + jl_inv(w) d."""
    w = np.asarray(w, dtype=np.float64)
    th2 = float(w @ w)
    th = np.sqrt(th2)
    K = hat(w)
    if th < SMALL:
        c = 1.0 / 12.0 + th2 / 720.0 + th2 * th2 / 30240.0
    else:
        c = 1.0 / th2 - (1.0 + np.cos(th)) / (2.0 * th * np.sin(th))
    return np.eye(3) - 0.5 * K + c * (K @ K)


def jr_inv(w):
    """Inverse right Jacobian: Log(Exp(w) Exp(d)) ~= w + jr_inv(w) d."""
    return jl_inv(-np.asarray(w, dtype=np.float64))


@dataclass
class State:
    """x = [r_WC, q_WC, v_IS (in I), b_g, b_a, q_IW] (Eq. 1)."""
    r: np.ndarray
    q: np.ndarray
    v: np.ndarray
    bg: np.ndarray
    ba: np.ndarray
    qg: np.ndarray

    @property
    def R(self):
        return quat_to_rot(self.q)

    @property
    def Rg(self):
        return quat_to_rot(self.qg)

    def copy(self):
        return State(self.r.copy(), self.q.copy(), self.v.copy(), self.bg.copy(),
                     self.ba.copy(), self.qg.copy())

    @staticmethod
    def from_dict(d):
        f = lambda k: np.array(d[k], dtype=np.float64)  # noqa: E731
        q = f("q_WC")
        qg = f("q_IW")
        return State(f("r_WC"), q / np.linalg.norm(q), f("v_I"), f("bg"), f("ba"),
                     qg / np.linalg.norm(qg))

    def to_dict(self):
        return dict(r_WC=self.r.copy(), q_WC=self.q.copy(), v_I=self.v.copy(),
                    bg=self.bg.copy(), ba=self.ba.copy(), q_IW=self.qg.copy())


def boxplus(x, d):
    """x boxplus dx (Eq. 2): vector parts add; q_WC <- exp(da) (x) q_WC;
    q_IW <- exp([dg_x, dg_y, 0]) (x) q_IW."""
    d = np.asarray(d, dtype=np.float64)
    q = quat_mul(quat_exp(d[3:6]), x.q)
    qg = quat_mul(quat_exp(np.array([d[15], d[16], 0.0])), x.qg)
    return State(x.r + d[0:3], q / np.linalg.norm(q), x.v + d[6:9], x.bg + d[9:12],
                 x.ba + d[12:15], qg / np.linalg.norm(qg))


def boxminus(x, y):
    """x boxminus y (Eq. 2): vector parts subtract; orientations log(p (x) q^-1);
    the gravity part keeps the x and y components of its log."""
    out = np.zeros(TANGENT_DIM)
    out[0:3] = x.r - y.r
    out[3:6] = quat_log(quat_mul(x.q, quat_conj(y.q)))
    out[6:9] = x.v - y.v
    out[9:12] = x.bg - y.bg
    out[12:15] = x.ba - y.ba
    out[15:17] = quat_log(quat_mul(x.qg, quat_conj(y.qg)))[0:2]
    return out
