"""Gauge invariance of the IMU term (Eq. 5, Sec. IV-C): gravity points along the
inertial frame's z axis, so turning the inertial frame about it -- q_IW and the
velocity v_I (expressed in I) rotated together by the same R_z -- changes no
measurement.  The position, rotation and bias rows of the IMU error stay,
the velocity and gravity rows turn with R_z, and the weighted cost e^T W e
(W recomputed at the turned x_0) stays.  A transposed R_IW or a gravity
vector taken in the wrong frame anywhere in the prediction fails this."""
import numpy as np
import pytest

from conftest import oracle_config
from oracle import imu
from oracle.so3 import State, boxplus, quat_mul, rot_to_quat
from paper_2207_10940_gb300 import synth


def _rz(a):
    c, s = np.cos(a), np.sin(a)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def _turn(x, Rz):
    y = x.copy()
    y.qg = quat_mul(rot_to_quat(Rz), x.qg)          # R_IW <- R_z R_IW
    y.v = Rz @ x.v
    return y


@pytest.mark.parametrize("angle", [0.3, -1.7, 3.0])
def test_turning_the_inertial_frame_about_gravity(angle):
    seq = synth.frame_pair(seed=6, cam=synth.scaled_camera(16, 12))
    cfg = oracle_config(seq)
    rng = np.random.default_rng(int(1000 * abs(angle)))
    x0 = boxplus(State.from_dict(seq.gt[0]), rng.normal(size=17) * 0.05)
    x1 = boxplus(State.from_dict(seq.gt[1]), rng.normal(size=17) * 0.05)
    t0, t1 = seq.frame_times
    pre = imu.preintegrate(seq.imu, t0, t1, x0.bg, x0.ba)
    e, _ = imu.residual(x0, x1, pre, cfg)
    W, _ = imu.weight(x0, seq.imu, t0, t1, cfg)
    Rz = _rz(angle)
    y0, y1 = _turn(x0, Rz), _turn(x1, Rz)
    f, _ = imu.residual(y0, y1, pre, cfg)
    Wy, _ = imu.weight(y0, seq.imu, t0, t1, cfg)
    scale = np.abs(e).max()
    for rows in (slice(0, 3), slice(3, 6), slice(9, 12), slice(12, 15)):
        np.testing.assert_allclose(f[rows], e[rows], atol=1e-12 * max(1.0, scale))
    np.testing.assert_allclose(f[6:9], Rz @ e[6:9], atol=1e-12 * max(1.0, scale))
    np.testing.assert_allclose(f[15:18], Rz @ e[15:18], atol=1e-12)
    c, cy = e @ W @ e, f @ Wy @ f
    assert abs(cy - c) <= 1e-9 * max(1.0, c), (c, cy)
    # the turn is not a no-op: the velocity error really moves
    assert np.linalg.norm(f[6:9] - e[6:9]) > 1e-3 * np.linalg.norm(e[6:9])


def test_turning_about_another_axis_is_seen():
    """The same turn about I's x axis tilts gravity: the IMU error changes."""
    seq = synth.frame_pair(seed=6, cam=synth.scaled_camera(16, 12))
    cfg = oracle_config(seq)
    x0, x1 = State.from_dict(seq.gt[0]), State.from_dict(seq.gt[1])
    t0, t1 = seq.frame_times
    pre = imu.preintegrate(seq.imu, t0, t1, x0.bg, x0.ba)
    e, _ = imu.residual(x0, x1, pre, cfg)
    c, s = np.cos(0.2), np.sin(0.2)
    Rx = np.array([[1.0, 0.0, 0.0], [0.0, c, -s], [0.0, s, c]])
    f, _ = imu.residual(_turn(x0, Rx), _turn(x1, Rx), pre, cfg)
    assert np.linalg.norm(f[0:3] - e[0:3]) > 1e-4
