"""Odometry accuracy of a tracked trajectory against ground truth.

This is the evaluation the paper reports for its tracker: the absolute
trajectory error of the camera positions (Sec. V, RMSE after a rigid
alignment) and how the estimated velocity and IMU biases converge to the true
ones (Fig. 3).  Here it runs on synthetic sequences whose ground truth is
exact.  Host-side numpy on the states the library returns; it evaluates
results and takes no part in tracking.

A state is a dict with r_WC (3), q_WC (w, x, y, z) or R_WC (3x3), v_I (3),
bg (3), ba (3), as returned by ``dri.state_to_dict`` and stored in a
sequence's ``gt`` list.  Both trajectories are expressed in the tracker's
world frame W (the first camera frame), so no alignment is needed for the
unaligned errors.
"""
from __future__ import annotations

import numpy as np


def _rot(s):
    if "R_WC" in s:
        return np.asarray(s["R_WC"], dtype=np.float64)
    w, x, y, z = (float(v) for v in s["q_WC"])
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def rotation_angle(R):
    """Angle of a rotation matrix, accurate near 0 and near pi (atan2 of the
    sine from the skew part and the cosine from the trace)."""
    R = np.asarray(R, dtype=np.float64)
    v = np.array([R[2, 1] - R[1, 2], R[0, 2] - R[2, 0], R[1, 0] - R[0, 1]])
    return float(np.arctan2(0.5 * np.linalg.norm(v), 0.5 * (np.trace(R) - 1.0)))


def align_rigid(est, gt):
    """Rotation R and translation t minimising sum |R est_i + t - gt_i|^2 (the
    closed form from the SVD of the cross-covariance of the centred point
    sets, without scale: monocular scale is not a gauge of RGB-D tracking)."""
    est = np.asarray(est, dtype=np.float64)
    gt = np.asarray(gt, dtype=np.float64)
    me, mg = est.mean(axis=0), gt.mean(axis=0)
    C = (gt - mg).T @ (est - me)
    U, _, Vt = np.linalg.svd(C)
    D = np.eye(3)
    D[2, 2] = np.sign(np.linalg.det(U @ Vt)) or 1.0
    R = U @ D @ Vt
    return R, mg - R @ me


def ate_rmse(est, gt, align=True):
    """Root mean square of the position errors, after the rigid alignment of
    the estimated positions onto the true ones when `align`."""
    est = np.asarray(est, dtype=np.float64)
    gt = np.asarray(gt, dtype=np.float64)
    if align:
        R, t = align_rigid(est, gt)
        est = est @ R.T + t
    return float(np.sqrt(np.mean(np.sum((est - gt) ** 2, axis=1))))


def evaluate(states, gt):
    """Errors of tracked states against ground truth, frame by frame.

    Returns a dict: ate_rmse_m (rigidly aligned) and ate_rmse_unaligned_m,
    final_position_error_m, rotation_rmse_rad, velocity_rmse_mps, and the final
    gyro / accelerometer bias errors (norms, rad/s and m/s^2) with their values
    at the first frame, the convergence the paper plots in Fig. 3."""
    n = len(states)
    if n == 0 or n != len(gt):
        raise ValueError("states and ground truth must be equally long and not empty")
    p = np.array([s["r_WC"] for s in states], dtype=np.float64)
    pg = np.array([g["r_WC"] for g in gt], dtype=np.float64)
    ang = np.array([rotation_angle(_rot(g).T @ _rot(s)) for s, g in zip(states, gt)])
    v = np.array([s["v_I"] for s in states], dtype=np.float64)
    vg = np.array([g["v_I"] for g in gt], dtype=np.float64)
    bg = np.array([np.linalg.norm(np.asarray(s["bg"]) - np.asarray(g["bg"])) for s, g in zip(states, gt)])
    ba = np.array([np.linalg.norm(np.asarray(s["ba"]) - np.asarray(g["ba"])) for s, g in zip(states, gt)])
    return {
        "frames": n,
        "ate_rmse_m": ate_rmse(p, pg, align=n >= 3),
        "ate_rmse_unaligned_m": ate_rmse(p, pg, align=False),
        "final_position_error_m": float(np.linalg.norm(p[-1] - pg[-1])),
        "rotation_rmse_rad": float(np.sqrt(np.mean(ang ** 2))),
        "velocity_rmse_mps": float(np.sqrt(np.mean(np.sum((v - vg) ** 2, axis=1)))),
        "bg_error_first": float(bg[0]), "bg_error_final": float(bg[-1]),
        "ba_error_first": float(ba[0]), "ba_error_final": float(ba[-1]),
    }
