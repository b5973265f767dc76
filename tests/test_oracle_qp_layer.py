"""Pins of the oracle's Step-1 QP layer (forward and vector-Jacobian product).

The layer is the learned sampler's optimization layer (Sec. IV): the convex
Step-1 QP of Alg. 1 line 7 as a function of p and of the initial state b0.
The adjoint formula of step1_layer_vjp is pinned by central finite
differences of the forward (the map is affine, so differences are exact up to
rounding) and by the dot-product identity <g, J v> = <J^T g, v>."""
import numpy as np
import pytest

from oracle import lower
from oracle.basis import bernstein
from paper_2212_02224_gb300 import scenegen as sg


def _setup(n_seg=1, m=60, n=11, B=5, seed=0):
    prm = sg.Params(m=m, n_coef=n, n_seg=n_seg)
    basis = bernstein(m, n, prm.dt)
    s = sg.Stream(seed)
    p = np.concatenate([s.uniform(0.0, 14.0, B * n_seg).reshape(B, n_seg),
                        s.uniform(5.0, 25.0, B * n_seg).reshape(B, n_seg)], axis=1)
    b0 = np.stack([s.uniform(-5, 5, B), s.uniform(0, 14, B), s.uniform(5, 20, B),
                   s.uniform(-1, 1, B), s.uniform(-2, 2, B), s.uniform(-1, 1, B)], axis=1)
    return prm, basis, p, b0


def test_layer_with_shared_state_is_step1():
    prm, sc, _ = sg.workload(0)
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    p = sg.make_samples(3, sc, 7, prm.n_seg)
    b0 = np.repeat(np.asarray(sc.ego, float)[None], 7, axis=0)
    np.testing.assert_allclose(lower.step1_layer(p, b0, prm, basis), lower.step1(p, sc, prm, basis),
                               rtol=1e-12, atol=1e-10)


@pytest.mark.parametrize("n_seg,n", [(1, 11), (4, 11), (2, 16)])
def test_vjp_matches_central_differences(n_seg, n):
    prm, basis, p, b0 = _setup(n_seg=n_seg, n=n, B=3, seed=n_seg * 10 + n)
    g = sg.Stream(5).normal(0.0, 1.0, 3 * 2 * n).reshape(3, 2 * n)
    gp, gb = lower.step1_layer_vjp(g, prm, basis)
    loss = lambda pp, bb: float(np.sum(g * lower.step1_layer(pp, bb, prm, basis)))
    h = 1e-3
    fd_p = np.zeros_like(p)
    for j in range(p.shape[0]):
        for a in range(p.shape[1]):
            e = np.zeros_like(p)
            e[j, a] = h
            fd_p[j, a] = (loss(p + e, b0) - loss(p - e, b0)) / (2 * h)
    fd_b = np.zeros_like(b0)
    for j in range(b0.shape[0]):
        for a in range(6):
            e = np.zeros_like(b0)
            e[j, a] = h
            fd_b[j, a] = (loss(p, b0 + e) - loss(p, b0 - e)) / (2 * h)
    np.testing.assert_allclose(gp, fd_p, rtol=1e-6, atol=1e-6 * np.abs(fd_p).max())
    np.testing.assert_allclose(gb, fd_b, rtol=1e-6, atol=1e-6 * np.abs(fd_b).max())


def test_dot_product_identity():
    prm, basis, p, b0 = _setup(n_seg=2, B=4, seed=9)
    s = sg.Stream(11)
    g = s.normal(0.0, 1.0, 4 * 2 * prm.n_coef).reshape(4, 2 * prm.n_coef)
    vp = s.normal(0.0, 1.0, p.size).reshape(p.shape)
    vb = s.normal(0.0, 1.0, b0.size).reshape(b0.shape)
    Jv = lower.step1_layer(p + vp, b0 + vb, prm, basis) - lower.step1_layer(p, b0, prm, basis)
    gp, gb = lower.step1_layer_vjp(g, prm, basis)
    lhs = np.sum(g * Jv)
    rhs = np.sum(gp * vp) + np.sum(gb * vb)
    assert abs(lhs - rhs) <= 1e-8 * max(1.0, abs(lhs))


def test_initial_state_gradient_of_a_position_loss():
    """A loss on the first position coefficient only: the first Bernstein
    coefficient equals x(0) (W[0] = e_0), so d c_x,0 / d x0 = 1 and the other
    entries of b0 do not move it."""
    prm, basis, p, b0 = _setup(B=2, seed=4)
    g = np.zeros((2, 2 * prm.n_coef))
    g[:, 0] = 1.0
    gp, gb = lower.step1_layer_vjp(g, prm, basis)
    np.testing.assert_allclose(gb[:, 0], 1.0, atol=1e-9)
    np.testing.assert_allclose(gb[:, 1:], 0.0, atol=1e-9)
    np.testing.assert_allclose(gp, 0.0, atol=1e-9)
