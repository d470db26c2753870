"""Pins of the oracle's inertial pre-integration and IMU term (Sec. IV-C, Eq. 5)."""
import numpy as np
import pytest

from conftest import oracle_config
from oracle import imu
from oracle.params import TrackerConfig
from oracle.so3 import State, boxplus, exp_so3, jr
from paper_2207_10940_gb300 import synth


def _samples(t, gyr, acc):
    t = np.asarray(t, dtype=np.float64)
    return np.column_stack([t, np.tile(gyr, (len(t), 1)), np.tile(acc, (len(t), 1))])


def test_pieces_cover_the_interval_and_reject_gaps():
    s = _samples(np.arange(0, 11) * 0.01, np.zeros(3), np.zeros(3))
    p = imu.pieces(s, 0.015, 0.052)
    assert p[0] == (1, pytest.approx(0.005))          # last sample with t <= t0
    assert sum(dt for _, dt in p) == pytest.approx(0.037, abs=1e-15)
    assert [k for k, _ in p] == [1, 2, 3, 4, 5]
    with pytest.raises(imu.CoverageError):
        imu.pieces(s, -0.001, 0.05)
    with pytest.raises(imu.CoverageError):
        imu.pieces(s, 0.02, 0.2)


def test_constant_rotation_rate_closed_form():
    """dR = Exp(w T) and d(dR)/d(b_g) = -Jr(w T) T for a constant rate."""
    w = np.array([0.3, -1.1, 0.7])
    s = _samples(np.arange(0, 40) / 200.0, w, np.zeros(3))
    T = 0.1234
    pre = imu.preintegrate(s, 0.0013, 0.0013 + T, np.zeros(3), np.zeros(3))
    np.testing.assert_allclose(pre["dR"], exp_so3(w * T), atol=1e-14)
    np.testing.assert_allclose(pre["Phi_g"], -jr(w * T) * T, atol=1e-14)


def test_constant_acceleration_closed_form():
    a = np.array([0.5, -2.0, 9.81])
    s = _samples(np.arange(0, 40) / 200.0, np.zeros(3), a)
    T = 0.0777
    pre = imu.preintegrate(s, 0.004, 0.004 + T, np.zeros(3), np.zeros(3))
    np.testing.assert_allclose(pre["dv"], a * T, atol=1e-15)
    np.testing.assert_allclose(pre["dp"], 0.5 * a * T * T, atol=1e-15)
    np.testing.assert_allclose(pre["P_a"], -0.5 * T * T * np.eye(3), atol=1e-15)
    np.testing.assert_allclose(pre["V_a"], -T * np.eye(3), atol=1e-15)


def test_stationary_imu_measures_gravity_reading():
    """At rest the accelerometer reads +g along I's up axis; the prediction then
    keeps position and velocity (Table I: g = 9.81)."""
    cfg = TrackerConfig(8, 8, 8, 8, 4, 4, levels=1, iters=(1,), R_CS=np.eye(3), r_CS=np.zeros(3))
    R_IW = exp_so3([0.2, -0.1, 0.4])
    from oracle.so3 import rot_to_quat
    x0 = State(np.array([1.0, 2.0, 3.0]), rot_to_quat(exp_so3([0.1, 0.2, -0.3])), np.zeros(3),
               np.zeros(3), np.zeros(3), rot_to_quat(R_IW))
    R_IS = R_IW @ x0.R
    f = R_IS.T @ np.array([0.0, 0.0, 9.81])
    s = _samples(np.arange(0, 30) / 200.0, np.zeros(3), f)
    pre = imu.preintegrate(s, 0.0, 0.1, np.zeros(3), np.zeros(3))
    pr = imu.predict(x0, pre, cfg)
    np.testing.assert_allclose(pr["r"], x0.r, atol=1e-14)
    np.testing.assert_allclose(pr["v"], 0.0, atol=1e-14)
    np.testing.assert_allclose(pr["R"], x0.R, atol=1e-14)


def test_residual_zero_at_ground_truth_zoh_exact():
    """Constant body rate + constant velocity make the zero-order hold exact, so
    e_IMU(GT) = 0 with noise-free samples (any biases, any extrinsic)."""
    for seed in (1, 2, 3):
        seq = synth.frame_pair(seed=seed, cam=synth.scaled_camera(16, 12), imu_noise=False)
        cfg = oracle_config(seq)
        x0, x1 = State.from_dict(seq.gt[0]), State.from_dict(seq.gt[1])
        pre = imu.preintegrate(seq.imu, seq.frame_times[0], seq.frame_times[1], x0.bg, x0.ba)
        e, _ = imu.residual(x0, x1, pre, cfg)
        assert np.max(np.abs(e)) < 1e-12


@pytest.fixture(scope="module")
def imu_case():
    seq = synth.frame_pair(seed=4, cam=synth.scaled_camera(16, 12))
    cfg = oracle_config(seq)
    rng = np.random.default_rng(21)
    x0 = boxplus(State.from_dict(seq.gt[0]), rng.normal(size=17) * 0.05)
    x1 = boxplus(State.from_dict(seq.gt[1]), rng.normal(size=17) * 0.05)
    return seq, cfg, x0, x1


def test_imu_jacobian_matches_finite_differences(imu_case):
    """All 18 x 34 entries, re-integrating at the perturbed biases."""
    seq, cfg, x0, x1 = imu_case
    t0, t1 = seq.frame_times

    def e_of(a, b):
        pre = imu.preintegrate(seq.imu, t0, t1, a.bg, a.ba)
        return imu.residual(a, b, pre, cfg)[0]

    pre = imu.preintegrate(seq.imu, t0, t1, x0.bg, x0.ba)
    J = imu.jacobian(x0, x1, pre, cfg)
    h = 1e-6
    for k in range(34):
        d = np.zeros(17)
        d[k % 17] = h
        if k < 17:
            fd = (e_of(boxplus(x0, d), x1) - e_of(boxplus(x0, -d), x1)) / (2 * h)
        else:
            fd = (e_of(x0, boxplus(x1, d)) - e_of(x0, boxplus(x1, -d))) / (2 * h)
        np.testing.assert_allclose(fd, J[:, k], atol=2e-8 * max(1.0, np.abs(J[:, k]).max()),
                                   err_msg=f"column {k}")


def test_bias_jacobians_of_preintegration(imu_case):
    seq, cfg, x0, _ = imu_case
    t0, t1 = seq.frame_times
    pre = imu.preintegrate(seq.imu, t0, t1, x0.bg, x0.ba)
    h = 1e-6
    for i in range(3):
        d = np.zeros(3)
        d[i] = h
        p = imu.preintegrate(seq.imu, t0, t1, x0.bg + d, x0.ba)
        m = imu.preintegrate(seq.imu, t0, t1, x0.bg - d, x0.ba)
        from oracle.so3 import log_so3
        dphi = (log_so3(pre["dR"].T @ p["dR"]) - log_so3(pre["dR"].T @ m["dR"])) / (2 * h)
        np.testing.assert_allclose(dphi, pre["Phi_g"][:, i], atol=1e-9)
        np.testing.assert_allclose((p["dv"] - m["dv"]) / (2 * h), pre["V_g"][:, i], atol=1e-9)
        np.testing.assert_allclose((p["dp"] - m["dp"]) / (2 * h), pre["P_g"][:, i], atol=1e-9)
        p = imu.preintegrate(seq.imu, t0, t1, x0.bg, x0.ba + d)
        m = imu.preintegrate(seq.imu, t0, t1, x0.bg, x0.ba - d)
        np.testing.assert_allclose((p["dv"] - m["dv"]) / (2 * h), pre["V_a"][:, i], atol=1e-9)
        np.testing.assert_allclose((p["dp"] - m["dp"]) / (2 * h), pre["P_a"][:, i], atol=1e-9)


def test_noise_propagation_matches_monte_carlo(imu_case):
    """Sigma_pre is the linear propagation of per-piece white noise
    (variance density^2 / dt); sampling that noise through the nonlinear
    recursion must give the same covariance (within sampling error)."""
    seq, cfg, x0, _ = imu_case
    t0, t1 = seq.frame_times
    gnd, and_ = 0.05, 0.5            # large densities so the test is not rounding-limited
    pre = imu.preintegrate(seq.imu, t0, t1, x0.bg, x0.ba, gnd, and_)
    pcs = imu.pieces(seq.imu, t0, t1)
    rng = np.random.default_rng(0)
    n = 4000
    out = np.zeros((n, 9))
    from oracle.so3 import log_so3
    for j in range(n):
        s = seq.imu.copy()
        for k, dt in pcs:
            s[k, 1:4] += rng.normal(0, gnd / np.sqrt(dt), 3)
            s[k, 4:7] += rng.normal(0, and_ / np.sqrt(dt), 3)
        q = imu.preintegrate(s, t0, t1, x0.bg, x0.ba)
        out[j, 0:3] = log_so3(pre["dR"].T @ q["dR"])
        out[j, 3:6] = q["dv"] - pre["dv"]
        out[j, 6:9] = q["dp"] - pre["dp"]
    C = np.cov(out.T)
    S = pre["Sigma"]
    sd = np.sqrt(np.diag(S))
    corr_err = np.abs(C - S) / np.outer(sd, sd)
    assert corr_err.max() < 0.12


def test_weight_symmetric_positive_definite(imu_case):
    seq, cfg, x0, _ = imu_case
    W, S = imu.weight(x0, seq.imu, *seq.frame_times, cfg)
    np.testing.assert_allclose(S, S.T, atol=1e-20)
    np.testing.assert_allclose(W @ S, np.eye(18), atol=1e-6)
    assert np.linalg.eigvalsh(S).min() > 0
