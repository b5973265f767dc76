"""Pins of the oracle's trajectory basis (Eq. param) against mathematics and
an independent library routine (scipy's Bernstein-polynomial evaluator)."""
import numpy as np
import pytest
from scipy.interpolate import BPoly

from oracle.basis import bernstein


@pytest.mark.parametrize("m,n", [(100, 11), (200, 16), (20, 6), (80, 11)])
def test_partition_of_unity_and_derivative_sums(m, n):
    W, Wd, Wdd = bernstein(m, n, 0.05)
    np.testing.assert_allclose(W.sum(1), 1.0, atol=1e-13)
    np.testing.assert_allclose(Wd.sum(1), 0.0, atol=1e-10)
    np.testing.assert_allclose(Wdd.sum(1), 0.0, atol=1e-8)
    assert (W >= 0).all()


@pytest.mark.parametrize("m,n", [(100, 11), (200, 16)])
def test_polynomial_reproduction(m, n):
    """Bernstein control points k/d reproduce tau; k(k-1)/(d(d-1)) reproduce tau^2."""
    dt = 0.05
    W, Wd, Wdd = bernstein(m, n, dt)
    d = n - 1
    tf = (m - 1) * dt
    tau = np.arange(m) / (m - 1)
    k = np.arange(n, dtype=float)
    c1 = k / d
    np.testing.assert_allclose(W @ c1, tau, atol=1e-13)
    np.testing.assert_allclose(Wd @ c1, 1.0 / tf, atol=1e-11)
    np.testing.assert_allclose(Wdd @ c1, 0.0, atol=1e-9)
    c2 = k * (k - 1) / (d * (d - 1))
    np.testing.assert_allclose(W @ c2, tau ** 2, atol=1e-13)
    np.testing.assert_allclose(Wd @ c2, 2 * tau / tf, atol=1e-11)
    np.testing.assert_allclose(Wdd @ c2, 2 / tf ** 2, atol=1e-9)


def test_against_scipy_bpoly():
    m, n, dt = 100, 11, 0.05
    W, Wd, Wdd = bernstein(m, n, dt)
    tf = (m - 1) * dt
    t = np.arange(m) * dt
    rng = np.random.default_rng(3)
    c = rng.normal(size=n) * 10
    bp = BPoly(c[:, None], [0.0, tf])
    np.testing.assert_allclose(W @ c, bp(t), rtol=1e-12, atol=1e-11)
    np.testing.assert_allclose(Wd @ c, bp.derivative(1)(t), rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(Wdd @ c, bp.derivative(2)(t), rtol=1e-9, atol=1e-9)


def test_finite_differences():
    m, n, dt = 400, 11, 0.0125
    W, Wd, Wdd = bernstein(m, n, dt)
    fd1 = (W[2:] - W[:-2]) / (2 * dt)
    fd2 = (W[2:] - 2 * W[1:-1] + W[:-2]) / dt ** 2
    np.testing.assert_allclose(fd1, Wd[1:-1], atol=2e-3 * np.abs(Wd).max())
    np.testing.assert_allclose(fd2, Wdd[1:-1], atol=2e-3 * np.abs(Wdd).max())
