"""Pins of the oracle's rotation and state-manifold code (Sec. IV-A, Eq. 1-2)."""
import numpy as np
import pytest
from scipy.linalg import expm, logm

from oracle import so3
from oracle.so3 import State, boxminus, boxplus


def _rand_state(rng):
    q = rng.normal(size=4)
    qg = rng.normal(size=4)
    return State(rng.normal(size=3), q / np.linalg.norm(q), rng.normal(size=3),
                 rng.normal(size=3) * 0.01, rng.normal(size=3) * 0.1, qg / np.linalg.norm(qg))


@pytest.mark.parametrize("scale", [1e-9, 1e-4, 1e-2, 0.5, 2.5])
def test_exp_matches_matrix_exponential(scale, rng):
    for _ in range(5):
        w = rng.normal(size=3) * scale
        np.testing.assert_allclose(so3.exp_so3(w), expm(so3.hat(w)), atol=1e-14)
        np.testing.assert_allclose(so3.quat_to_rot(so3.quat_exp(w)), expm(so3.hat(w)), atol=1e-14)


@pytest.mark.parametrize("scale", [1e-9, 1e-4, 0.3, 2.0])
def test_log_inverts_exp(scale, rng):
    for _ in range(5):
        w = rng.normal(size=3) * scale
        n = np.linalg.norm(w)
        if n > 3.0:                       # log returns the rotation angle in [0, pi)
            w *= 3.0 / n
        np.testing.assert_allclose(so3.log_so3(so3.exp_so3(w)), w, atol=1e-13, rtol=1e-10)
        np.testing.assert_allclose(so3.quat_log(so3.quat_exp(w)), w, atol=1e-14, rtol=1e-12)
    w = rng.normal(size=3) * scale
    R = so3.exp_so3(w * min(1.0, 3.0 / np.linalg.norm(w)))
    np.testing.assert_allclose(so3.hat(so3.log_so3(R)), np.real(logm(R)), atol=1e-10)


def test_hamilton_product_composes_rotations(rng):
    for _ in range(10):
        p = rng.normal(size=4)
        q = rng.normal(size=4)
        p /= np.linalg.norm(p)
        q /= np.linalg.norm(q)
        np.testing.assert_allclose(so3.quat_to_rot(so3.quat_mul(p, q)),
                                   so3.quat_to_rot(p) @ so3.quat_to_rot(q), atol=1e-14)
    # Hamilton convention: i * j = k
    np.testing.assert_allclose(so3.quat_mul([0, 1, 0, 0], [0, 0, 1, 0]), [0, 0, 0, 1])


@pytest.mark.parametrize("scale", [1e-5, 0.2, 1.5])
def test_se3_jacobians_against_finite_differences(scale, rng):
    h = 1e-6
    for _ in range(3):
        w = rng.normal(size=3) * scale
        w *= min(1.0, 2.8 / np.linalg.norm(w))      # stay inside the log's domain
        Jr = so3.jr(w)
        Jli = so3.jl_inv(w)
        Jri = so3.jr_inv(w)
        for i in range(3):
            d = np.zeros(3)
            d[i] = h
            # Exp(w + d) = Exp(w) Exp(Jr d)
            fd = (so3.log_so3(so3.exp_so3(w).T @ so3.exp_so3(w + d))
                  - so3.log_so3(so3.exp_so3(w).T @ so3.exp_so3(w - d))) / (2 * h)
            np.testing.assert_allclose(fd, Jr[:, i], atol=1e-8)
            # Log(Exp(d) Exp(w)) = w + Jl^-1 d
            fd = (so3.log_so3(so3.exp_so3(d) @ so3.exp_so3(w))
                  - so3.log_so3(so3.exp_so3(-d) @ so3.exp_so3(w))) / (2 * h)
            np.testing.assert_allclose(fd, Jli[:, i], atol=1e-8)
            fd = (so3.log_so3(so3.exp_so3(w) @ so3.exp_so3(d))
                  - so3.log_so3(so3.exp_so3(w) @ so3.exp_so3(-d))) / (2 * h)
            np.testing.assert_allclose(fd, Jri[:, i], atol=1e-8)


def test_boxplus_boxminus_invariants(rng):
    """(x boxplus d) boxminus x = d for every tangent direction (Eq. 2)."""
    for _ in range(20):
        x = _rand_state(rng)
        d = rng.normal(size=17) * 0.3
        np.testing.assert_allclose(boxminus(boxplus(x, d), x), d, atol=1e-14, rtol=1e-12)
        np.testing.assert_allclose(boxminus(x, x), np.zeros(17), atol=1e-15)


def test_boxplus_of_difference_recovers_state(rng):
    """x boxplus (y boxminus x) = y whenever y differs from x inside the
    parameterised directions (the gravity yaw gauge is held fixed)."""
    for _ in range(20):
        x = _rand_state(rng)
        y = boxplus(x, rng.normal(size=17) * 0.5)
        z = boxplus(x, boxminus(y, x))
        for a, b in [(z.r, y.r), (z.v, y.v), (z.bg, y.bg), (z.ba, y.ba)]:
            np.testing.assert_allclose(a, b, atol=1e-14)
        np.testing.assert_allclose(z.R, y.R, atol=1e-14)
        np.testing.assert_allclose(z.Rg, y.Rg, atol=1e-14)


def test_orientation_perturbation_is_global():
    """q boxplus da = exp(da) (x) q: a perturbation about W's z turns W-frame
    vectors, not camera-frame ones."""
    q = so3.quat_exp(np.array([0.0, np.pi / 2, 0.0]))
    x = State(np.zeros(3), q, np.zeros(3), np.zeros(3), np.zeros(3), np.array([1.0, 0, 0, 0]))
    d = np.zeros(17)
    d[5] = 0.1
    y = boxplus(x, d)
    np.testing.assert_allclose(y.R, so3.exp_so3([0, 0, 0.1]) @ x.R, atol=1e-15)
