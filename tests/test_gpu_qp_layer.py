"""The differentiable Step-1 layer through the C ABI: forward and backward
against the oracle (float64, same bar as the FP64 path), and torch's
finite-difference gradient check of the autograd wrapper on the GPU."""
import numpy as np
import pytest
import torch

from oracle import lower
from oracle.basis import bernstein
from paper_2212_02224_gb300 import binding, scenegen as sg

from gpu_common import FP64_XI_REL, planner, to_dev

pytestmark = pytest.mark.gpu


def _inputs(prm, B, seed):
    s = sg.Stream(seed)
    ns = prm.n_seg
    p = np.concatenate([s.uniform(0.0, 14.0, B * ns).reshape(B, ns),
                        s.uniform(5.0, 25.0, B * ns).reshape(B, ns)], axis=1)
    b0 = np.stack([s.uniform(-5, 5, B), s.uniform(0, 14, B), s.uniform(5, 20, B),
                   s.uniform(-1, 1, B), s.uniform(-2, 2, B), s.uniform(-1, 1, B)], axis=1)
    return p, b0


def _rel(a, b):
    return np.abs(a - b).max() / max(1.0, np.abs(b).max())


@pytest.mark.parametrize("n_seg,n,m,B", [(1, 11, 100, 1), (1, 11, 100, 1000), (4, 11, 100, 37),
                                         (2, 16, 200, 65), (1, 8, 37, 5)])
def test_forward_and_backward_match_oracle(n_seg, n, m, B):
    prm = sg.Params(m=m, n_coef=n, n_seg=n_seg)
    basis = bernstein(m, n, prm.dt)
    p, b0 = _inputs(prm, B, seed=B + n)
    g = sg.Stream(3).normal(0.0, 1.0, B * 2 * n).reshape(B, 2 * n)
    pl = planner(prm, "fp64", max_obs=1, max_samples=B)
    xi = pl.qp_forward(to_dev(p), to_dev(b0)).cpu().numpy()
    gp, gb = pl.qp_backward(to_dev(g))
    gp_only, none = pl.qp_backward(to_dev(g), want_b0=False)
    torch.cuda.synchronize()
    pl.close()
    assert _rel(xi, lower.step1_layer(p, b0, prm, basis)) <= FP64_XI_REL
    op, ob = lower.step1_layer_vjp(g, prm, basis)
    assert _rel(gp.cpu().numpy(), op) <= FP64_XI_REL
    assert _rel(gb.cpu().numpy(), ob) <= FP64_XI_REL
    assert none is None and torch.equal(gp_only, gp)


def test_forward_with_shared_state_is_the_solve_prologue():
    """With b0 = the scene's ego state the layer is Step 1 of the solve: the
    FP64 solve with zero projection iterations would start from it; compare
    with the oracle's step1 of the scene."""
    prm, sc, _ = sg.workload(1)
    p = sg.make_samples(5, sc, 40, prm.n_seg)
    b0 = np.repeat(np.asarray(sc.ego, float)[None], 40, axis=0)
    pl = planner(prm, "fp32", max_obs=16, max_samples=40)
    xi = pl.qp_forward(to_dev(p), to_dev(b0)).cpu().numpy()
    pl.close()
    ref = lower.step1(p, sc, prm, bernstein(prm.m, prm.n_coef, prm.dt))
    assert _rel(xi, ref) <= FP64_XI_REL


def test_autograd_gradcheck():
    prm = sg.Params(n_seg=2)
    pl = planner(prm, "fp32", max_obs=1, max_samples=8)
    p, b0 = _inputs(prm, 3, seed=17)
    tp = to_dev(p).requires_grad_()
    tb = to_dev(b0).requires_grad_()
    assert torch.autograd.gradcheck(lambda a, b: pl.qp_layer(a, b), (tp, tb), eps=1e-3,
                                    atol=1e-7, rtol=1e-7)
    pl.close()


def test_layer_fits_set_points_by_gradient_descent():
    """A use of the layer: recover the set-points that produced a target
    trajectory by gradient descent on the squared coefficient error."""
    prm = sg.Params(n_seg=1)
    pl = planner(prm, "fp32", max_obs=1, max_samples=16)
    p_true, b0 = _inputs(prm, 16, seed=23)
    target = pl.qp_forward(to_dev(p_true), to_dev(b0)).detach()
    p = (to_dev(p_true) + 2.0).requires_grad_()
    tb = to_dev(b0)
    opt = torch.optim.Adam([p], lr=0.5)
    first = None
    for _ in range(300):
        opt.zero_grad()
        loss = ((pl.qp_layer(p, tb) - target) ** 2).sum()
        loss.backward()
        opt.step()
        first = first if first is not None else float(loss.detach())
    pl.close()
    assert float(loss.detach()) < 1e-4 * first
    assert np.abs(p.detach().cpu().numpy() - p_true).max() < 0.05


def test_capacity_and_null_errors():
    prm = sg.Params()
    pl = planner(prm, "fp32", max_obs=1, max_samples=4)
    p, b0 = _inputs(prm, 5, seed=1)
    with pytest.raises(binding.PlanError) as e:
        pl.qp_forward(to_dev(p), to_dev(b0))
    assert e.value.status == binding.PLAN_ECAPACITY
    with pytest.raises(binding.PlanError) as e:
        binding.plan_qp_backward(pl.ctx, 0, 2, 0, 0)
    assert e.value.status == binding.PLAN_EINVAL
    pl.close()
