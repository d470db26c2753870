"""Pins of the oracle's gyro-only variant (track_mode 2: the tracker with the
accelerometer-related IMU residuals ignored, Sec. VII, Fig. 5 and Table VI)."""
import numpy as np
import pytest

from conftest import oracle_config
from oracle import gn, imu
from oracle.so3 import State, log_so3
from paper_2207_10940_gb300 import synth

KEPT = imu.GYRO_ROWS
DROPPED = np.setdiff1d(np.arange(18), KEPT)


def _tracker(seq, levels=2, iters=(6, 4), **kw):
    cfg = oracle_config(seq, levels=levels, iters=iters, track_mode=2, **kw)
    tr = gn.Tracker(cfg, synth.initial_state(seq))
    tr.push_imu(seq.imu)
    tr.track(seq.depth[0], seq.intensity[0], seq.frame_times[0])
    return tr, cfg


@pytest.fixture(scope="module")
def pair():
    return synth.frame_pair(seed=3, cam=synth.scaled_camera(64, 48))


def test_weight_is_the_information_left_on_the_kept_rows(pair):
    """Dropping residual rows leaves the inverse of their covariance block, which
    is the Schur complement of the full information over the dropped rows."""
    cfg = oracle_config(pair)
    x0 = State.from_dict(synth.initial_state(pair))
    t0, t1 = pair.frame_times
    W, S = imu.weight(x0, pair.imu, t0, t1, cfg)
    Wg = imu.weight_gyro_only(S)
    assert not Wg[DROPPED].any() and not Wg[:, DROPPED].any()
    K, D = np.ix_(KEPT, KEPT), np.ix_(DROPPED, DROPPED)
    schur = W[K] - W[np.ix_(KEPT, DROPPED)] @ np.linalg.solve(W[D], W[np.ix_(DROPPED, KEPT)])
    np.testing.assert_allclose(Wg[K], schur, rtol=1e-7, atol=1e-7 * np.abs(schur).max())
    # the kept rows' noise comes from the gyroscope alone
    cfg_a = oracle_config(pair, acc_nd=10 * cfg.acc_nd, acc_rw=10 * cfg.acc_rw)
    _, S_a = imu.weight(x0, pair.imu, t0, t1, cfg_a)
    assert np.array_equal(imu.weight_gyro_only(S_a), Wg)
    assert not np.allclose(S_a, S)


def test_accelerometer_samples_do_not_matter(pair):
    """The accelerometer readings reach only the dropped rows, whose weight is
    zero: replacing them changes no bit of the result."""
    rng = np.random.default_rng(8)
    bad = pair.imu.copy()
    bad[:, 4:7] = rng.normal(scale=5.0, size=(len(bad), 3))
    out = []
    for samples in (pair.imu, bad):
        cfg = oracle_config(pair, levels=2, iters=(5, 3), track_mode=2)
        tr = gn.Tracker(cfg, synth.initial_state(pair))
        tr.push_imu(samples)
        tr.track(pair.depth[0], pair.intensity[0], pair.frame_times[0])
        out.append(tr.track(pair.depth[1], pair.intensity[1], pair.frame_times[1]))
    a, b = out
    for f in ("r", "q", "v", "bg", "ba", "qg"):
        assert np.array_equal(getattr(a["x1"], f), getattr(b["x1"], f)), f
    assert np.array_equal(a["H"], b["H"]) and np.array_equal(a["H_prior"], b["H_prior"])


def test_held_components_stay_and_carry_no_prior(pair):
    tr, _ = _tracker(pair)
    x0 = tr.x.copy()
    r = tr.track(pair.depth[1], pair.intensity[1], pair.frame_times[1])
    for f in ("v", "ba"):
        assert np.array_equal(getattr(r["x1"], f), getattr(x0, f)), f
    # the gravity quaternion is renormalised by every state update
    np.testing.assert_allclose(r["x1"].qg, x0.qg, rtol=0, atol=1e-15)
    held = gn.HELD_GYRO_ONLY
    assert not r["H_prior"][held].any() and not r["H_prior"][:, held].any()
    assert not r["b_prior"][held].any()
    free = np.setdiff1d(np.arange(17), held)
    assert np.all(np.linalg.eigvalsh(r["H_prior"][np.ix_(free, free)]) > 0)
    # the gyro bias is estimated: it moves
    assert not np.array_equal(r["x1"].bg, x0.bg)


def test_held_system_solves_the_system_without_the_held_components(pair):
    """Identity rows for the held components equal deleting them (the step on
    the others is the reduced system's solution; theirs is zero)."""
    tr, cfg = _tracker(pair)
    from oracle.maps import frame_levels
    lv = frame_levels(pair.depth[1], pair.intensity[1], cfg)
    x0 = tr.x.copy()
    t0, t1 = tr.t, pair.frame_times[1]
    _, S = imu.weight(x0, tr.imu, t0, t1, cfg)
    Wg = imu.weight_gyro_only(S)
    x1 = x0.copy()
    H, b, _ = tr.linearise_all(lv, 0, x0, x1, t0, t1, Wg)
    cfg.track_mode = 0                       # the same terms, nothing held
    Hf, bf, _ = tr.linearise_all(lv, 0, x0, x1, t0, t1, Wg)
    cfg.track_mode = 2
    held = np.r_[gn.HELD_GYRO_ONLY, 17 + gn.HELD_GYRO_ONLY]
    free = np.setdiff1d(np.arange(34), held)
    d = gn.cholesky_solve(H, b)
    d_red = gn.cholesky_solve(Hf[np.ix_(free, free)], bf[free])
    assert not d[held].any()
    # the pose prior (1e12) against the bias information makes the system's
    # condition number ~1e12: the two factorisations round apart by ~1e-8
    np.testing.assert_allclose(d[free], d_red, rtol=1e-6, atol=1e-12)


def test_converges_to_the_true_motion_noise_free():
    seq = synth.frame_pair(seed=3, cam=synth.scaled_camera(96, 72), sigma_d=0.0, sigma_I=0.0,
                           imu_noise=False)
    tr, _ = _tracker(seq, iters=(8, 5))
    r = tr.track(seq.depth[1], seq.intensity[1], seq.frame_times[1])
    g = State.from_dict(seq.gt[1])
    assert np.linalg.norm(log_so3(r["x1"].R @ g.R.T)) < 2e-3
    assert np.linalg.norm(r["x1"].r - g.r) < 5e-3


def test_first_iterate_is_the_gyro_rotation_prediction(pair):
    """x_1 starts at x_0's position and velocity, rotated by the pre-integrated
    gyro rotation: R_WC0 R_CS dR R_CS^T (the camera's rotation over the frame
    seen from the IMU)."""
    tr, cfg = _tracker(pair)
    rng = np.random.default_rng(2)
    x0 = tr.x.copy()
    x0.bg = x0.bg + rng.normal(scale=0.01, size=3)
    t0, t1 = tr.t, pair.frame_times[1]
    pre = imu.preintegrate(tr.imu, t0, t1, x0.bg, x0.ba)
    x1 = tr.first_iterate(x0, pre)
    for f in ("r", "v", "bg", "ba", "qg"):
        assert np.array_equal(getattr(x1, f), getattr(x0, f)), f
    R_pred = x0.R @ cfg.R_CS @ pre["dR"] @ cfg.R_CS.T
    assert np.linalg.norm(log_so3(x1.R @ R_pred.T)) < 1e-14
    # the ground-truth rotation over the frame, to the gyro noise over 1/30 s
    g0, g1 = State.from_dict(pair.gt[0]), State.from_dict(pair.gt[1])
    ours = R_pred @ x0.R.T
    truth = g1.R @ g0.R.T
    assert np.linalg.norm(log_so3(ours @ truth.T)) < 2e-3
