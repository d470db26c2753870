"""Pins of the oracle's cost, Gauss-Newton system, prior and marginalisation (Eq. 6-9)."""
import json
import os

import numpy as np
import pytest

from conftest import oracle_config
from oracle import gn, imu, params
from oracle.so3 import State, boxminus, boxplus, log_so3
from paper_2207_10940_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_table1_constants():
    t = json.load(open(os.path.join(GOLDEN, "table1_synthetic.json")))
    assert params.GYR_NOISE_DENSITY == t["gyr_noise_density"]
    assert params.ACC_NOISE_DENSITY == t["acc_noise_density"]
    assert params.GYR_BIAS_PRIOR == t["gyr_bias_prior"]
    assert params.ACC_BIAS_PRIOR == t["acc_bias_prior"]
    assert params.GYR_DRIFT_DENSITY == t["gyr_drift_noise_density"]
    assert params.ACC_DRIFT_DENSITY == t["acc_drift_noise_density"]
    assert params.GRAVITY == t["gravity_m_s2"]
    assert params.IMU_RATE == t["imu_rate_hz"]


def _spd(rng, n, cond=1e6):
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    return Q @ np.diag(np.logspace(0, np.log10(cond), n)) @ Q.T


def test_schur_complement_equals_marginal_information():
    """Eq. 8 is the information form of marginalising a Gaussian: H* equals the
    inverse of the x_1 block of H^-1 and H*^-1 b* its mean (textbook identity)."""
    rng = np.random.default_rng(0)
    for _ in range(5):
        H = _spd(rng, 34)
        b = rng.normal(size=34)
        Hs, bs = gn.schur(H, b)
        C = np.linalg.inv(H)
        np.testing.assert_allclose(Hs, np.linalg.inv(C[17:, 17:]), rtol=1e-8,
                                   atol=1e-10 * np.abs(Hs).max())
        np.testing.assert_allclose(np.linalg.solve(Hs, bs), (C @ b)[17:], rtol=1e-8, atol=1e-10)


def test_prior_only_step_lands_on_prior_mean():
    """With only Eq. 6's prior term, one step from any x_0 that differs from
    xbar_0 in its vector parts lands exactly on xbar_0 boxplus H*^-1 b*."""
    rng = np.random.default_rng(1)
    xbar = State(rng.normal(size=3), np.array([1.0, 0, 0, 0]), rng.normal(size=3),
                 rng.normal(size=3) * 0.01, rng.normal(size=3) * 0.1, np.array([1.0, 0, 0, 0]))
    d = np.zeros(17)
    d[[0, 1, 2, 6, 7, 8, 9, 10, 11, 12, 13, 14]] = rng.normal(size=12)
    x0 = boxplus(xbar, d)
    Hs = _spd(rng, 17, 1e4)
    bs = rng.normal(size=17)
    Hp, bp = gn.prior_terms(x0, xbar, Hs, bs)
    step = np.linalg.solve(Hp, bp)
    want = np.linalg.solve(Hs, bs)
    np.testing.assert_allclose(boxminus(boxplus(x0, step), xbar), want, atol=1e-12)


@pytest.fixture(scope="module")
def imu_prior_case():
    seq = synth.frame_pair(seed=5, cam=synth.scaled_camera(16, 12))
    cfg = oracle_config(seq)
    rng = np.random.default_rng(4)
    x0 = boxplus(State.from_dict(seq.gt[0]), rng.normal(size=17) * 0.03)
    x1 = boxplus(State.from_dict(seq.gt[1]), rng.normal(size=17) * 0.03)
    # prior mean differs from x_0 only in the vector parts (the reading's
    # identity Jacobian of x_0 boxminus xbar_0 is then exact)
    dv = np.zeros(17)
    dv[[0, 1, 2, 6, 7, 8, 9, 10, 11, 12, 13, 14]] = rng.normal(size=12) * 0.02
    xbar = boxplus(x0, dv)
    Hs = _spd(rng, 17, 1e3) * 100
    bs = rng.normal(size=17) * 10
    return seq, cfg, x0, x1, xbar, Hs, bs


def test_gradient_of_cost_is_minus_two_b(imu_prior_case):
    """FD gradient of Eq. 6's IMU + prior terms, evaluated directly from their
    definition, equals -2 b of the assembled system (Eq. 7)."""
    seq, cfg, x0, x1, xbar, Hs, bs = imu_prior_case
    t0, t1 = seq.frame_times
    W, _ = imu.weight(x0, seq.imu, t0, t1, cfg)
    zero = dict(H_rgb=np.zeros((12, 12)), b_rgb=np.zeros(12), H_icp=np.zeros((6, 6)),
                b_icp=np.zeros(6))

    def cost(a, b_):
        pre = imu.preintegrate(seq.imu, t0, t1, a.bg, a.ba)
        e, _ = imu.residual(a, b_, pre, cfg)
        return float(e @ W @ e) + gn.prior_cost(a, xbar, Hs, bs)

    pre = imu.preintegrate(seq.imu, t0, t1, x0.bg, x0.ba)
    e, pr = imu.residual(x0, x1, pre, cfg)
    J = imu.jacobian(x0, x1, pre, cfg, e, pr)
    H, b = gn.assemble(zero, J, e, W, x0, xbar, Hs, bs)
    h = 1e-6
    g = np.zeros(34)
    for k in range(34):
        d = np.zeros(17)
        d[k % 17] = h
        if k < 17:
            g[k] = (cost(boxplus(x0, d), x1) - cost(boxplus(x0, -d), x1)) / (2 * h)
        else:
            g[k] = (cost(x0, boxplus(x1, d)) - cost(x0, boxplus(x1, -d))) / (2 * h)
    np.testing.assert_allclose(g, -2 * b, rtol=2e-6, atol=1e-6 * np.abs(b).max())
    np.testing.assert_allclose(H, H.T, rtol=1e-12, atol=1e-12 * np.abs(H).max())


def _run_pair(seq, cfg, x_init, x1_override=None):
    tr = gn.Tracker(cfg, x_init)
    tr.push_imu(seq.imu)
    tr.track(seq.depth[0], seq.intensity[0], seq.frame_times[0])
    return tr, tr.track(seq.depth[1], seq.intensity[1], seq.frame_times[1])


def test_gn_converges_and_step_vanishes(pair_small):
    cfg = oracle_config(pair_small, iters=(12, 6))
    tr, res = _run_pair(pair_small, cfg, synth.initial_state(pair_small))
    assert res["status"] == "ok"
    step = np.abs(res["d_last"])
    assert step[:6].max() < 1e-7 and step[17:23].max() < 1e-7
    gt = pair_small.gt[1]
    x1 = res["x1"]
    assert np.linalg.norm(x1.r - gt["r_WC"]) < 0.01
    assert np.linalg.norm(log_so3(x1.R @ gt["R_WC"].T)) < np.deg2rad(1.0)
    # marginal prior is symmetric positive definite
    Hs = res["H_prior"]
    np.testing.assert_allclose(Hs, Hs.T, rtol=1e-9, atol=1e-9 * np.abs(Hs).max())
    assert np.linalg.eigvalsh(Hs).min() > 0


def test_gn_fixed_point_independent_of_start(pair_small):
    """Starting x_1 away from the IMU prediction (~1 deg, 2 cm) reaches the same
    fixed point as the default start."""
    cfg = oracle_config(pair_small, iters=(15, 8))
    xi = synth.initial_state(pair_small)
    _, ref = _run_pair(pair_small, cfg, xi)
    tr = gn.Tracker(cfg, xi)
    tr.push_imu(pair_small.imu)
    tr.track(pair_small.depth[0], pair_small.intensity[0], pair_small.frame_times[0])
    orig = gn.imu_mod.predict

    def shifted(x0, pre, c):
        out = orig(x0, pre, c)
        from oracle.so3 import exp_so3
        out = dict(out)
        out["R"] = exp_so3([0.01, -0.012, 0.008]) @ out["R"]
        out["r"] = out["r"] + np.array([0.015, -0.01, 0.01])
        return out

    gn.imu_mod.predict = shifted
    try:
        # only the initialisation uses the shifted prediction: restore it after
        # the first call through a one-shot wrapper
        calls = {"n": 0}

        def once(x0, pre, c):
            calls["n"] += 1
            return shifted(x0, pre, c) if calls["n"] == 1 else orig(x0, pre, c)

        gn.imu_mod.predict = once
        res = tr.track(pair_small.depth[1], pair_small.intensity[1], pair_small.frame_times[1])
    finally:
        gn.imu_mod.predict = orig
    np.testing.assert_allclose(res["x1"].r, ref["x1"].r, atol=2e-5)
    assert np.linalg.norm(log_so3(res["x1"].R @ ref["x1"].R.T)) < 2e-5


def test_sequence_chaining_keeps_tracking():
    seq = synth.sinusoid_sequence(seed=3, cam=synth.scaled_camera(96, 72), n_frames=4)
    cfg = oracle_config(seq, levels=2, iters=(6, 4))
    tr = gn.Tracker(cfg, synth.initial_state(seq))
    tr.push_imu(seq.imu)
    for i in range(4):
        res = tr.track(seq.depth[i], seq.intensity[i], seq.frame_times[i])
        if i:
            gt = seq.gt[i]
            assert np.linalg.norm(res["x1"].r - gt["r_WC"]) < 0.03
            assert np.linalg.norm(log_so3(res["x1"].R @ gt["R_WC"].T)) < np.deg2rad(2.0)


def test_cholesky_failure_reports_lost(pair_small):
    cfg = oracle_config(pair_small)
    tr = gn.Tracker(cfg, synth.initial_state(pair_small))
    tr.push_imu(pair_small.imu)
    tr.track(pair_small.depth[0], pair_small.intensity[0], pair_small.frame_times[0])
    tr.Hs = -np.eye(17)            # an indefinite prior makes H indefinite
    with pytest.raises(gn.TrackingLost):
        tr.track(pair_small.depth[1], pair_small.intensity[1], pair_small.frame_times[1])
