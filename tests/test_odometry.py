"""Pins of the odometry metrics (paper Sec. V absolute trajectory error, Fig. 3
convergence): closed forms and invariants, no GPU."""
import numpy as np

from paper_2207_10940_gb300 import odometry


def _rz(a):
    c, s = np.cos(a), np.sin(a)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def _random_rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def test_rigid_alignment_recovers_a_rigid_motion():
    rng = np.random.default_rng(3)
    gt = rng.normal(size=(40, 3))
    R, t = _random_rotation(rng), rng.normal(size=3)
    est = (gt - t) @ R                       # gt = R est + t
    Ra, ta = odometry.align_rigid(est, gt)
    assert np.allclose(Ra, R, atol=1e-12) and np.allclose(ta, t, atol=1e-12)
    assert odometry.ate_rmse(est, gt) < 1e-12
    assert odometry.ate_rmse(est, gt, align=False) > 0.1


def test_alignment_is_proper_for_planar_points():
    # coplanar points: the SVD's third direction is arbitrary; a reflection must
    # not be returned
    gt = np.array([[1.0, 0, 0], [0, 1, 0], [-1, 0, 0], [0, -1, 0], [0.5, 0.5, 0]])
    est = gt @ _rz(0.4).T
    R, _ = odometry.align_rigid(est, gt)
    assert np.isclose(np.linalg.det(R), 1.0) and odometry.ate_rmse(est, gt) < 1e-12


def test_constant_offset_and_symmetric_noise_closed_forms():
    gt = np.array([[1.0, 0, 0], [0, 1, 0], [-1, 0, 0], [0, -1, 0]])
    d = np.array([0.3, -0.4, 1.2])
    assert np.isclose(odometry.ate_rmse(gt + d, gt, align=False), 1.3)
    assert odometry.ate_rmse(gt + d, gt) < 1e-12
    # radial errors +e, -e, +e, -e on a square: the best rigid motion is the
    # identity by symmetry, so the aligned error is e
    e = 0.01
    est = gt * (1 + e * np.array([1, -1, 1, -1]))[:, None]
    assert np.isclose(odometry.ate_rmse(est, gt), e, rtol=1e-9)


def test_rotation_angle():
    for a in (1e-9, 1e-4, 0.3, 2.0, 3.1):
        assert np.isclose(odometry.rotation_angle(_rz(a)), a, rtol=1e-9, atol=1e-15)


def test_evaluate_on_ground_truth_and_a_perturbed_copy():
    rng = np.random.default_rng(5)
    gt = []
    for k in range(10):
        R = _rz(0.1 * k)
        gt.append(dict(r_WC=rng.normal(size=3), R_WC=R, v_I=rng.normal(size=3),
                       bg=np.full(3, 1e-3), ba=np.full(3, 0.05)))
    ev = odometry.evaluate(gt, gt)
    assert ev["ate_rmse_m"] < 1e-12 and ev["rotation_rmse_rad"] < 1e-12
    assert ev["velocity_rmse_mps"] == 0.0 and ev["bg_error_final"] == 0.0
    est = [dict(g, r_WC=g["r_WC"] + [0.0, 0.0, 0.02], R_WC=g["R_WC"] @ _rz(0.01),
                v_I=g["v_I"] + [0.1, 0.0, 0.0], bg=np.zeros(3), ba=g["ba"] + [0.0, 0.03, 0.04])
           for g in gt]
    ev = odometry.evaluate(est, gt)
    assert np.isclose(ev["ate_rmse_unaligned_m"], 0.02) and ev["ate_rmse_m"] < 1e-12
    assert np.isclose(ev["rotation_rmse_rad"], 0.01)
    assert np.isclose(ev["velocity_rmse_mps"], 0.1)
    assert np.isclose(ev["bg_error_final"], np.sqrt(3) * 1e-3)
    assert np.isclose(ev["ba_error_final"], 0.05)
