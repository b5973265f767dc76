"""Parity of the goal-parameterised lower level and outer loop through the C ABI
against the FP64 oracle: p = [y_d.., v_d.., x_f, y_f] (Eq. behaviour_param)
with the final rows (x(t_f), y(t_f), ydot(t_f)) = (x_f, y_f, 0) of
Eq. final_boundary in A_eq xi = b(p) (Eq. lower_eq).  Every path (plain FP64,
fused FP32, tensor-core TF32X3), the first-iteration sampler, whole Alg. 1
cycles and the Step-1 layer."""
import numpy as np
import pytest
import torch

from oracle import lower, upper
from oracle.basis import bernstein
from paper_2212_02224_gb300 import scenegen as sg

from gpu_common import FP32_POS_M, compare, planner, position_error, to_dev

pytestmark = pytest.mark.gpu


def _goal_prm(**kw):
    prm, sc, B = sg.workload(1, goal=True, **kw)
    return prm, sc, B


def _samples(seed, sc, prm, B):
    return sg.make_samples(seed, sc, B, prm.n_seg, goal_tf=(prm.m - 1) * prm.dt)


def _run(prec, prm, sc, p, shape=None):
    pl = planner(prm, prec, max_obs=max(sc.n_obs, 1), max_samples=len(p))
    if shape:
        pl.set_tuning(*shape)
    xi, r, cu = pl.solve(sc, to_dev(p))
    torch.cuda.synchronize()
    out = xi.cpu().numpy(), r.cpu().numpy(), cu.cpu().numpy()
    pl.close()
    return out


def _oracle(prm, sc, p):
    return lower.solve(p, sc, prm, bernstein(prm.m, prm.n_coef, prm.dt))


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3"])
@pytest.mark.parametrize("n_seg", [1, 4])
def test_goal_dense_traffic_parity(prec, n_seg):
    """Dense-traffic scene, 100 iterations, 72 samples with goals."""
    prm, sc, _ = _goal_prm(n_seg=n_seg)
    p = _samples(404 + n_seg, sc, prm, 72)
    out = _run(prec, prm, sc, p)
    if prec == "tf32x3":
        # split-TF32 products are float32-level: the FP32 bar applies
        compare("fp32", prm, *out, *_oracle(prm, sc, p), sc=sc, p=p)
    else:
        compare(prec, prm, *out, *_oracle(prm, sc, p), sc=sc, p=p)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-8), ("fp32", FP32_POS_M)])
def test_goal_rows_met_by_gpu_plans(prec, tol):
    """The returned plans end at their goal with zero lateral velocity."""
    prm, sc, _ = _goal_prm(inner_iters=60)
    p = _samples(9, sc, prm, 50)
    xi, _, _ = _run(prec, prm, sc, p)
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    n = prm.n_coef
    W, Wd = basis[0][-1], basis[1][-1]
    np.testing.assert_allclose(xi[:, :n] @ W, p[:, 2], atol=tol)
    np.testing.assert_allclose(xi[:, n:] @ W, p[:, 3], atol=tol)
    np.testing.assert_allclose(xi[:, n:] @ Wd, 0.0, atol=tol)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_goal_full_batch(prec):
    """B = 1000 goal samples solved together, every one compared with the oracle."""
    prm, sc, B = _goal_prm()
    p = _samples(505, sc, prm, B)
    out = compare(prec, prm, *_run(prec, prm, sc, p), *_oracle(prm, sc, p), sc=sc, p=p)
    # a goal far short of the set-point speeds makes a few samples brake hard
    # through the traffic; their outcome bifurcates under float32 rounding
    assert out.get("ill_conditioned", 0) <= 5


@pytest.mark.parametrize("shape", [(1, 8), (2, 2), (4, 1)])
def test_goal_fused_shapes(shape):
    prm, sc, _ = _goal_prm(inner_iters=40, n_seg=2)
    p = _samples(606, sc, prm, 40)
    compare("fp32", prm, *_run("fp32", prm, sc, p, shape), *_oracle(prm, sc, p), sc=sc, p=p)


def test_goal_wide_basis_long_horizon():
    """n = 16, m = 200 (the scale workload's basis and horizon) with goals."""
    prm, sc, _ = sg.workload(4, inner_iters=40, goal=True)
    p = _samples(707, sc, prm, 24)
    for prec in ("fp64", "fp32"):
        compare(prec, prm, *_run(prec, prm, sc, p), *_oracle(prm, sc, p), sc=sc, p=p)


def test_goal_sampler_matches_oracle_draws():
    prm = sg.Params(n_seg=4, goal=True, m=100)
    sc = sg.make_scene(3, n_lanes=4, n_obs=0)
    sc.ego[0] = 1.5
    pl = planner(prm, "fp32", max_obs=1, max_samples=3000)
    B = 3000
    p_fresh = pl.sample(sc, B, l=1, seed=0xABCDEF12345, step=3).cpu().numpy()
    np.testing.assert_allclose(p_fresh, upper.draw_initial(B, sc, prm, 0xABCDEF12345, 3),
                               rtol=1e-15, atol=1e-12)
    d = prm.d_p
    mu = np.linspace(1.0, 40.0, d)
    A = np.tril(np.full((d, d), 0.2)) + np.eye(d)
    sigma = A @ A.T
    p_g = pl.sample(sc, B, l=2, seed=5, step=1, mu=mu, sigma=sigma).cpu().numpy()
    pl.close()
    np.testing.assert_allclose(p_g, upper.draw_gaussian(B, mu, sigma, prm, 2, 5, 1), rtol=1e-12,
                               atol=1e-12)


def test_goal_mpc_cycle_fp64_matches_oracle():
    """A whole Alg. 1 cycle with goal entries (d_p = 4) on the FP64 path."""
    prm, sc, B = sg.workload(0, inner_iters=30, outer_iters=3, goal=True)
    pl = planner(prm, "fp64", max_obs=max(sc.n_obs, 1), max_samples=B)
    res = pl.step(sc, B, seed=33)
    pl.close()
    ref = upper.plan(sc, prm, B, seed=33)
    assert res["index"] == ref["best"]
    np.testing.assert_allclose(res["p"], ref["p"], rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(res["xi"], ref["xi"], rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(res["mu"], ref["mu"], rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(res["sigma"], ref["sigma"], rtol=1e-5, atol=1e-6)


def test_goal_mpc_cycle_fp32_four_segments():
    """d_p = 10 (four set-points per axis and the goal): the FP32 cycle returns
    a valid lower-level solution of its own p within the FP32 bar."""
    prm, sc, B = sg.workload(1, inner_iters=40, outer_iters=3, goal=True, n_seg=4)
    B = 400
    pl = planner(prm, "fp32", max_obs=sc.n_obs, max_samples=B)
    res = pl.step(sc, B, seed=12)
    pl.close()
    assert len(res["p"]) == 10 and len(res["mu"]) == 10
    xo, ro, co = _oracle(prm, sc, np.array([res["p"]]))
    assert position_error(np.array([res["xi"]]), xo, prm) <= FP32_POS_M
    assert abs(res["cost"] - (co[0] + ro[0])) <= 1e-4 * abs(co[0] + ro[0]) + 1e-3


def test_goal_qp_layer_matches_oracle():
    prm = sg.Params(m=60, n_coef=11, n_seg=2, goal=True)
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    s = sg.Stream(8)
    B = 16
    p = np.concatenate([s.uniform(0.0, 14.0, B * 2).reshape(B, 2), s.uniform(5.0, 25.0, B * 2).reshape(B, 2),
                        s.uniform(20.0, 70.0, B)[:, None], s.uniform(0.0, 14.0, B)[:, None]], axis=1)
    b0 = np.stack([s.uniform(-5, 5, B), s.uniform(0, 14, B), s.uniform(5, 20, B),
                   s.uniform(-1, 1, B), s.uniform(-2, 2, B), s.uniform(-1, 1, B)], axis=1)
    g = s.normal(0.0, 1.0, B * 2 * prm.n_coef).reshape(B, 2 * prm.n_coef)
    pl = planner(prm, "fp64", max_obs=1, max_samples=B)
    xi = pl.qp_forward(to_dev(p), to_dev(b0)).cpu().numpy()
    gp, gb = pl.qp_backward(to_dev(g))
    gp, gb = gp.cpu().numpy(), gb.cpu().numpy()
    pl.close()
    np.testing.assert_allclose(xi, lower.step1_layer(p, b0, prm, basis), rtol=1e-9, atol=1e-8)
    gp_o, gb_o = lower.step1_layer_vjp(g, prm, basis)
    np.testing.assert_allclose(gp, gp_o, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(gb, gb_o, rtol=1e-9, atol=1e-9)


def test_goal_needs_enough_coefficients():
    from paper_2212_02224_gb300 import binding
    prm = sg.Params(n_coef=5, goal=True)
    with pytest.raises(binding.PlanError) as e:
        planner(prm, "fp64", max_obs=1, max_samples=8)
    assert e.value.status == binding.PLAN_EINVAL
