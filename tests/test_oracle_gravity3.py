"""Pins of the oracle's 3-D gravity-with-gauge form of the state (gravity3.py,
Sec. II and IV-A: q_IW perturbed about all three axes, Levenberg-Marquardt
damping on the gravity blocks)."""
import numpy as np
import pytest

from conftest import oracle_config
from oracle import gn, gravity3, imu
from oracle.so3 import State, boxplus, hat, log_so3
from paper_2207_10940_gb300 import synth

EZ = np.array([0.0, 0.0, 1.0])


@pytest.fixture(scope="module")
def case():
    seq = synth.frame_pair(seed=4, cam=synth.scaled_camera(16, 12))
    cfg = oracle_config(seq)
    rng = np.random.default_rng(21)
    x0 = boxplus(State.from_dict(seq.gt[0]), rng.normal(size=17) * 0.05)
    x1 = boxplus(State.from_dict(seq.gt[1]), rng.normal(size=17) * 0.05)
    return seq, cfg, x0, x1


def test_boxplus_boxminus_round_trips(case):
    _, _, x0, x1 = case
    rng = np.random.default_rng(3)
    for scale in (1e-6, 1e-2, 0.5):
        d = rng.normal(size=18) * scale
        np.testing.assert_allclose(gravity3.boxminus(gravity3.boxplus(x0, d), x0), d,
                                   rtol=1e-10, atol=1e-14)
    y = gravity3.boxplus(x0, gravity3.boxminus(x1, x0))
    for f in ("r", "v", "bg", "ba"):
        np.testing.assert_allclose(getattr(y, f), getattr(x1, f), atol=1e-14)
    assert np.linalg.norm(log_so3(y.R @ x1.R.T)) < 1e-14
    assert np.linalg.norm(log_so3(y.Rg @ x1.Rg.T)) < 1e-14


def test_two_dof_form_is_the_three_dof_form_without_the_gauge_axis(case):
    _, _, x0, _ = case
    d = np.random.default_rng(5).normal(size=17) * 0.1
    a = boxplus(x0, d)
    b = gravity3.boxplus(x0, np.concatenate([d, [0.0]]))
    for f in ("r", "q", "v", "bg", "ba", "qg"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f


def test_jacobian_matches_finite_differences_and_the_two_dof_columns(case):
    seq, cfg, x0, x1 = case
    t0, t1 = seq.frame_times
    pre = imu.preintegrate(seq.imu, t0, t1, x0.bg, x0.ba)
    J = gravity3.imu_jacobian(x0, x1, pre, cfg)
    J2 = imu.jacobian(x0, x1, pre, cfg)
    keep3 = np.r_[0:17, 18:35]                       # drop the two gauge-axis columns
    assert np.array_equal(J[:, keep3], J2)

    def e_of(a, b):
        return imu.residual(a, b, imu.preintegrate(seq.imu, t0, t1, a.bg, a.ba), cfg)[0]

    h = 1e-6
    for k in range(36):
        d = np.zeros(18)
        d[k % 18] = h
        if k < 18:
            fd = (e_of(gravity3.boxplus(x0, d), x1) - e_of(gravity3.boxplus(x0, -d), x1)) / (2 * h)
        else:
            fd = (e_of(x0, gravity3.boxplus(x1, d)) - e_of(x0, gravity3.boxplus(x1, -d))) / (2 * h)
        np.testing.assert_allclose(fd, J[:, k], atol=2e-8 * max(1.0, np.abs(J[:, k]).max()),
                                   err_msg=f"column {k}")


def test_gauge_direction(case):
    """Turning the inertial frame about gravity (dg = e_z and dv = e_z x v on
    both states) moves the IMU error only by turning its velocity and gravity
    rows: J n = (0, 0, e_z x e_v, 0, 0, e_z x e_g)."""
    seq, cfg, x0, x1 = case
    t0, t1 = seq.frame_times
    pre = imu.preintegrate(seq.imu, t0, t1, x0.bg, x0.ba)
    e, _ = imu.residual(x0, x1, pre, cfg)
    J = gravity3.imu_jacobian(x0, x1, pre, cfg)
    n = np.zeros(36)
    n[6:9], n[15:18] = hat(EZ) @ x0.v, EZ
    n[24:27], n[33:36] = hat(EZ) @ x1.v, EZ
    want = np.zeros(18)
    want[6:9] = np.cross(EZ, e[6:9])
    want[15:18] = np.cross(EZ, e[15:18])
    np.testing.assert_allclose(J @ n, want, atol=1e-12 * max(1.0, np.abs(J).max()))
    # a turn about another axis tilts gravity: the velocity error moves by
    # about g T per radian (0.33 m/s over 1/30 s)
    nx = n.copy()
    nx[15:18] = nx[33:36] = [1.0, 0.0, 0.0]
    nx[6:9], nx[24:27] = hat([1.0, 0.0, 0.0]) @ x0.v, hat([1.0, 0.0, 0.0]) @ x1.v
    assert np.linalg.norm((J @ nx)[6:9]) > 0.1


def _track(seq, tracker):
    tracker.push_imu(seq.imu)
    tracker.track(seq.depth[0], seq.intensity[0], seq.frame_times[0])
    return tracker.track(seq.depth[1], seq.intensity[1], seq.frame_times[1])


def test_tracks_a_pair_like_the_two_dof_form():
    """Both forms reach the same camera poses.  Velocity and gravity direction
    in the world frame (R_IW^T v_I, R_IW^T e_z) agree far inside the priors'
    uncertainty: the priors are set on v_I and q_IW in each form's own
    parameterisation (the 3-D form's also on the turn about gravity), so the
    two costs differ slightly there.  The q_IW difference is mostly that turn,
    the gauge the 2-DoF form holds fixed.  The 3-D prior carries information
    on all three gravity axes."""
    seq = synth.frame_pair(seed=3, cam=synth.scaled_camera(64, 48))
    cfg = oracle_config(seq, levels=2, iters=(8, 5))
    a = _track(seq, gn.Tracker(cfg, synth.initial_state(seq)))["x1"]
    res = _track(seq, gravity3.Tracker(cfg, synth.initial_state(seq)))
    b = res["x1"]
    g = State.from_dict(seq.gt[1])
    assert np.linalg.norm(log_so3(a.R @ b.R.T)) < 1e-6
    assert np.linalg.norm(a.r - b.r) < 1e-6
    s = cfg.prior_sigma
    assert np.linalg.norm(a.Rg.T @ a.v - b.Rg.T @ b.v) < 1e-2 * s["v"]
    assert np.linalg.norm(a.Rg.T @ EZ - b.Rg.T @ EZ) < 1e-1 * s["grav"]
    err_a = np.linalg.norm(a.Rg.T @ a.v - g.Rg.T @ g.v)
    err_b = np.linalg.norm(b.Rg.T @ b.v - g.Rg.T @ g.v)
    assert abs(err_a - err_b) < 1e-2 * err_a
    turn = log_so3(b.Rg @ a.Rg.T)
    assert abs(turn[2]) > np.linalg.norm(turn[:2])
    Hs = res["H_prior"]
    assert Hs.shape == (18, 18) and np.all(np.linalg.eigvalsh(0.5 * (Hs + Hs.T)) > 0)


def test_damping_changes_the_path_not_the_minimum():
    seq = synth.frame_pair(seed=3, cam=synth.scaled_camera(64, 48))
    cfg = oracle_config(seq, levels=2, iters=(12, 8))
    res = [_track(seq, gravity3.Tracker(cfg, synth.initial_state(seq), damping=mu))
           for mu in (0.0, 1.0, 10.0)]
    for r in res[1:]:
        assert np.linalg.norm(log_so3(r["x1"].R @ res[0]["x1"].R.T)) < 1e-7
        assert np.linalg.norm(r["x1"].r - res[0]["x1"].r) < 1e-7
        assert np.linalg.norm(log_so3(r["x1"].Rg @ res[0]["x1"].Rg.T)) < 1e-6
