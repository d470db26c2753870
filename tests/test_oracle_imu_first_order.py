"""Pins of the first-order bias update of the pre-integration (Forster et al.,
the alternative to re-integrating at every Gauss-Newton iteration, imu_mode 1)."""
import numpy as np
import pytest

from conftest import oracle_config
from oracle import gn, imu
from oracle.so3 import State, boxplus, log_so3
from paper_2207_10940_gb300 import synth


@pytest.fixture(scope="module")
def case():
    seq = synth.frame_pair(seed=4, cam=synth.scaled_camera(16, 12))
    cfg = oracle_config(seq)
    rng = np.random.default_rng(21)
    x0 = boxplus(State.from_dict(seq.gt[0]), rng.normal(size=17) * 0.05)
    x1 = boxplus(State.from_dict(seq.gt[1]), rng.normal(size=17) * 0.05)
    return seq, cfg, x0, x1


def _gap(a, b):
    return (np.linalg.norm(log_so3(a["dR"].T @ b["dR"])) + np.linalg.norm(a["dv"] - b["dv"])
            + np.linalg.norm(a["dp"] - b["dp"]))


def test_update_is_exact_at_zero_and_for_the_accelerometer_bias(case):
    seq, _, x0, _ = case
    t0, t1 = seq.frame_times
    pre = imu.preintegrate(seq.imu, t0, t1, x0.bg, x0.ba)
    same = imu.correct(pre, np.zeros(3), np.zeros(3))
    for k in ("dR", "dv", "dp", "Phi_g", "V_g", "P_g", "V_a", "P_a"):
        assert np.array_equal(same[k], pre[k]), k
    # dv and dp are linear in b_a (the rotations do not depend on it)
    dba = np.array([0.3, -0.2, 0.1])
    ref = imu.preintegrate(seq.imu, t0, t1, x0.bg, x0.ba + dba)
    up = imu.correct(pre, np.zeros(3), dba)
    assert _gap(up, ref) < 1e-13


def test_update_error_is_second_order_in_the_gyro_bias(case):
    seq, _, x0, _ = case
    t0, t1 = seq.frame_times
    pre = imu.preintegrate(seq.imu, t0, t1, x0.bg, x0.ba)
    u = np.array([0.6, -0.48, 0.64])
    errs = []
    for eps in (0.4, 0.2, 0.1):
        ref = imu.preintegrate(seq.imu, t0, t1, x0.bg + eps * u, x0.ba)
        errs.append(_gap(imu.correct(pre, eps * u, np.zeros(3)), ref))
    for a, b in zip(errs, errs[1:]):
        assert 3.2 < a / b < 4.8, errs


def test_jacobian_of_the_updated_model_matches_finite_differences(case):
    """All 18 x 34 entries of the IMU term built on the updated pre-integration,
    away from the linearisation point (Jr(Phi_g dbg) differs from I)."""
    seq, cfg, x0, x1 = case
    t0, t1 = seq.frame_times
    bg0, ba0 = x0.bg.copy(), x0.ba.copy()
    pre0 = imu.preintegrate(seq.imu, t0, t1, bg0, ba0)
    xa = x0.copy()
    xa.bg = bg0 + np.array([0.3, -0.2, 0.25])
    xa.ba = ba0 + np.array([0.05, 0.02, -0.04])

    def e_of(a, b):
        return imu.residual(a, b, imu.correct(pre0, a.bg - bg0, a.ba - ba0), cfg)[0]

    J = imu.jacobian(xa, x1, imu.correct(pre0, xa.bg - bg0, xa.ba - ba0), cfg)
    h = 1e-6
    for k in range(34):
        d = np.zeros(17)
        d[k % 17] = h
        if k < 17:
            fd = (e_of(boxplus(xa, d), x1) - e_of(boxplus(xa, -d), x1)) / (2 * h)
        else:
            fd = (e_of(xa, boxplus(x1, d)) - e_of(xa, boxplus(x1, -d))) / (2 * h)
        np.testing.assert_allclose(fd, J[:, k], atol=2e-8 * max(1.0, np.abs(J[:, k]).max()),
                                   err_msg=f"column {k}")


def _track_pair(mode, **kw):
    seq = synth.frame_pair(seed=3, cam=synth.scaled_camera(64, 48))
    cfg = oracle_config(seq, levels=2, iters=(6, 4), imu_mode=mode, **kw)
    tr = gn.Tracker(cfg, synth.initial_state(seq))
    tr.push_imu(seq.imu)
    tr.track(seq.depth[0], seq.intensity[0], seq.frame_times[0])
    return tr.track(seq.depth[1], seq.intensity[1], seq.frame_times[1])


def test_tracker_first_order_mode():
    exact = _track_pair(0)
    first = _track_pair(1)
    # biases move by ~1e-2 within the frame: the update's error is second order
    assert np.linalg.norm(log_so3(exact["x1"].R @ first["x1"].R.T)) < 1e-6
    assert np.linalg.norm(exact["x1"].r - first["x1"].r) < 1e-6
    # re-integrating whenever the biases move reproduces the exact mode bit for bit
    always = _track_pair(1, bias_relin_g=0.0, bias_relin_a=0.0)
    assert np.array_equal(always["x1"].r, exact["x1"].r) and np.array_equal(always["H"], exact["H"])
