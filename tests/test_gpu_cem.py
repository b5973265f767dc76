"""Parity of the Alg. 1 stages (sampling, elite selection, distribution update)
and of whole MPC cycles through the C ABI against the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import lower, upper
from oracle.basis import bernstein
from paper_2212_02224_gb300 import binding, scenegen as sg

from gpu_common import FP32_POS_M, planner, positions, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("B,n_c,q,ties", [(1, 1, 1, False), (7, 5, 2, True), (1000, 150, 50, True),
                                          (1000, 150, 50, False), (5000, 2048, 700, True),
                                          (40000, 150, 50, True), (64, 64, 64, True),
                                          (2048, 1024, 300, False), (2048, 1000, 1000, True),
                                          (2049, 1024, 300, False), (100, 40, 10, "group"),
                                          (1500, 400, 120, True), (300, 256, 100, False),
                                          (257, 257, 3, True)])
def test_select_elites_bit_exact(B, n_c, q, ties):
    s = sg.Stream(B * 31 + n_c)
    if ties == "group":
        # exactly n_c zeros: the prefix group of the n_c-th key is taken whole
        r = np.concatenate([np.zeros(n_c), s.uniform(0.5, 3.0, B - n_c)])
        r = r[np.argsort(s.uniform(0.0, 1.0, B))]
        cu = s.uniform(100.0, 2000.0, B)
    elif ties:
        r = s.integers(0, 6, B).astype(float) * 0.25      # many exact ties, many zeros
        cu = s.integers(0, 9, B).astype(float)
    else:
        r = s.uniform(0.0, 3.0, B)
        cu = s.uniform(100.0, 2000.0, B)
    prm = sg.Params()
    pl = planner(prm, "fp32", max_obs=1, max_samples=16)
    el = pl.select_elites(to_dev(r), to_dev(cu), n_c, q).cpu().numpy()
    pl.close()
    C = upper.select_lowest(r, n_c)
    E = upper.select_lowest(cu + r, q, among=C)
    assert list(el) == list(E)


@pytest.mark.parametrize("case", ["near_equal_zero_path", "near_equal_sort_path", "signed_zeros",
                                  "nan_inf", "negative_costs"])
def test_select_elites_key_edge_cases(case):
    """Keys the selection must order exactly: costs equal in their upper 32
    bits (the EliteSet rank count compares those first), -0 against +0 (the
    same key), NaN after +inf, negative costs; with at least n_c zero scores
    (compaction path) and with fewer (sort path)."""
    B, n_c, q = 1000, 150, 50
    s = sg.Stream(sum(map(ord, case)))
    if case.startswith("near_equal"):
        # 1000 + j 2^-40: the doubles differ only in their lowest mantissa bits
        cu = 1000.0 + s.integers(0, 64, B).astype(float) * 2.0 ** -40
        n_zero = 400 if case.endswith("zero_path") else 100
        r = np.where(np.arange(B) < n_zero, 0.0, s.uniform(0.1, 2.0, B))
        r = r[np.argsort(s.uniform(0.0, 1.0, B))]
    elif case == "signed_zeros":
        r = np.where(s.uniform(0.0, 1.0, B) < 0.5, 0.0, -0.0)
        r[s.integers(0, B - 1, 200)] = 0.25
        cu = s.integers(0, 5, B).astype(float)
        cu[::7] = -0.0
    elif case == "nan_inf":
        r = s.integers(0, 3, B).astype(float) * 0.5
        r[s.integers(0, B - 1, 30)] = np.nan
        r[s.integers(0, B - 1, 30)] = np.inf
        cu = s.uniform(0.0, 10.0, B)
        cu[s.integers(0, B - 1, 30)] = np.nan
        cu[s.integers(0, B - 1, 30)] = np.inf
    else:
        r = s.integers(0, 3, B).astype(float)
        cu = s.uniform(-50.0, 50.0, B)
    prm = sg.Params()
    pl = planner(prm, "fp32", max_obs=1, max_samples=16)
    el = pl.select_elites(to_dev(r), to_dev(cu), n_c, q).cpu().numpy()
    pl.close()
    C = upper.select_lowest(r, n_c)
    E = upper.select_lowest(cu + r, q, among=C)
    assert list(el) == list(E)


def test_update_distribution():
    prm = sg.Params(n_seg=2, eta=0.7, gamma=0.9)
    s = sg.Stream(5)
    q = 50
    pe = s.normal(0.0, 3.0, q * 4).reshape(q, 4) + np.array([1.0, 5.0, 12.0, 20.0])
    cost = s.uniform(300.0, 320.0, q)
    mu = np.array([2.0, 4.0, 15.0, 18.0])
    A = s.normal(0.0, 1.0, 16).reshape(4, 4)
    sigma = A @ A.T + np.eye(4)
    mu_o, sg_o = upper.update_distribution(mu, sigma, pe, cost, prm)
    pl = planner(prm, "fp32", max_obs=1, max_samples=16)
    mu_t, sg_t = to_dev(mu), to_dev(sigma)
    pl.update_distribution(to_dev(pe), to_dev(cost), mu_t, sg_t)
    torch.cuda.synchronize()
    pl.close()
    np.testing.assert_allclose(mu_t.cpu().numpy(), mu_o, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(sg_t.cpu().numpy(), sg_o, rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("n_seg,q,offset,mu_shift", [(1, 1, 0.0, 3.0), (4, 50, 1.0e4, 250.0),
                                                   (4, 500, -30.0, 0.0), (2, 33, 5.0e3, -1.0e3)])
def test_update_distribution_shapes(n_seg, q, offset, mu_shift):
    """The update at d_p = 2 .. 8, one elite, many elites, an elite cloud far
    from the origin and a previous mean far from the cloud, against the
    oracle's two-pass Eqs. mean_update and cov_update."""
    prm = sg.Params(n_seg=n_seg, eta=0.6, gamma=0.9)
    d = prm.d_p
    s = sg.Stream(q * 7 + d)
    centre = offset + np.arange(d, dtype=float)
    pe = s.normal(0.0, 2.0, q * d).reshape(q, d) + centre
    cost = s.uniform(300.0, 330.0, q)
    mu = centre + mu_shift
    A = s.normal(0.0, 1.0, d * d).reshape(d, d)
    sigma = A @ A.T + np.eye(d)
    mu_o, sg_o = upper.update_distribution(mu, sigma, pe, cost, prm)
    pl = planner(prm, "fp32", max_obs=1, max_samples=16)
    mu_t, sg_t = to_dev(mu), to_dev(sigma)
    pl.update_distribution(to_dev(pe), to_dev(cost), mu_t, sg_t)
    torch.cuda.synchronize()
    pl.close()
    np.testing.assert_allclose(mu_t.cpu().numpy(), mu_o, rtol=1e-12, atol=1e-12)
    scale = np.abs(sg_o).max()
    np.testing.assert_allclose(sg_t.cpu().numpy(), sg_o, rtol=1e-11, atol=1e-12 * scale)


@pytest.mark.parametrize("n_seg", [1, 2, 4])
def test_sampler_matches_oracle_draws(n_seg):
    prm = sg.Params(n_seg=n_seg)
    sc = sg.make_scene(3, n_lanes=4, n_obs=0)
    pl = planner(prm, "fp32", max_obs=1, max_samples=3000)
    B = 3000
    p_fresh = pl.sample(sc, B, l=1, seed=0x1234ABCD5678, step=7).cpu().numpy()
    np.testing.assert_array_equal(p_fresh, upper.draw_initial(B, sc, prm, 0x1234ABCD5678, 7))
    d = 2 * n_seg
    mu = np.linspace(1.0, 20.0, d)
    A = np.tril(np.full((d, d), 0.3)) + np.eye(d)
    sigma = A @ A.T
    p_g = pl.sample(sc, B, l=3, seed=99, step=2, mu=mu, sigma=sigma).cpu().numpy()
    pl.close()
    p_o = upper.draw_gaussian(B, mu, sigma, prm, 3, 99, 2)
    np.testing.assert_allclose(p_g, p_o, rtol=1e-12, atol=1e-12)


def _cycle(prec, prm, sc, B, seed, step=0, mu=None, sigma=None):
    pl = planner(prm, prec, max_obs=max(sc.n_obs, 1), max_samples=B)
    res = pl.step(sc, B, mu=mu, sigma=sigma, seed=seed, step=step)
    pl.close()
    return res


def test_mpc_cycle_fp64_matches_oracle():
    """One full Alg. 1 cycle on the plain FP64 path equals the oracle's."""
    prm, sc, B = sg.workload(0, inner_iters=30, outer_iters=3)
    res = _cycle("fp64", prm, sc, B, seed=21)
    ref = upper.plan(sc, prm, B, seed=21)
    assert res["index"] == ref["best"]
    np.testing.assert_allclose(res["p"], ref["p"], rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(res["xi"], ref["xi"], rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(res["cost"], ref["cost"], rtol=1e-6)
    np.testing.assert_allclose(res["mu"], ref["mu"], rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(res["sigma"], ref["sigma"], rtol=1e-5, atol=1e-6)
    assert res["step"] == 1


def test_mpc_cycle_fp64_warm_start_matches_oracle():
    prm, sc, B = sg.workload(0, inner_iters=25, outer_iters=2)
    mu = np.array([4.0, 19.0])
    sigma = np.array([[2.0, 0.3], [0.3, 9.0]])
    res = _cycle("fp64", prm, sc, B, seed=8, step=5, mu=mu, sigma=sigma)
    ref = upper.plan(sc, prm, B, seed=8, step=5, mu=mu, sigma=sigma)
    assert res["index"] == ref["best"]
    np.testing.assert_allclose(res["mu"], ref["mu"], rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(res["cost"], ref["cost"], rtol=1e-6)


def test_mpc_cycle_fp32():
    """FP32 cycle: the returned pair is a valid lower-level solution of its own p
    (checked by the oracle) and its cost is close to the oracle's cycle."""
    prm, sc, B = sg.workload(0, inner_iters=30, outer_iters=3)
    res = _cycle("fp32", prm, sc, B, seed=21)
    ref = upper.plan(sc, prm, B, seed=21)
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    xo, ro, co = lower.solve(np.array([res["p"]]), sc, prm, basis)
    xg, yg = positions(np.array([res["xi"]]), prm)
    xr, yr = positions(xo, prm)
    assert float(np.hypot(xg - xr, yg - yr).max()) <= FP32_POS_M
    assert abs(res["cost"] - (co[0] + ro[0])) <= 1e-4 * abs(co[0] + ro[0]) + 1e-3
    assert res["cost"] <= ref["cost"] * 1.05 + 1e-3


def test_resident_graph_replay_is_deterministic():
    prm, sc, B = sg.workload(0, inner_iters=20, outer_iters=2)
    pl = planner(prm, "fp32", max_obs=8, max_samples=B)
    outs = []
    for _ in range(2):
        pl.upload([sc])
        pl.set_state(0, seed=3, step=0)
        pl.step_resident([B])
        outs.append((pl.get_result(0), pl.get_state(0)))
    pl.close()
    assert outs[0][0] == outs[1][0]
    assert outs[0][1]["mu"] == outs[1][1]["mu"]


def test_batched_scene_cycles_match_single_scene_cycles():
    """Scenes planned together give the same result as each planned alone."""
    prm, scenes, Bs = sg.batched_workload(S=4, seed=31, B_range=(20, 90), N_range=(2, 12),
                                          inner_iters=20, outer_iters=2)
    pl = planner(prm, "fp32", max_obs=16, max_samples=sum(Bs), max_scenes=4)
    pl.upload(scenes)
    for i in range(4):
        pl.set_state(i, seed=100 + i)
    pl.step_resident(Bs)
    together = [pl.get_result(i) for i in range(4)]
    alone = []
    for i in range(4):
        pl.upload([scenes[i]])
        pl.set_state(0, seed=100 + i)
        pl.step_resident([Bs[i]])
        alone.append(pl.get_result(0))
    pl.close()
    for a, b in zip(together, alone):
        assert a == b


def test_step_errors():
    prm, sc, B = sg.workload(0, inner_iters=5, outer_iters=1)
    pl = planner(prm, "fp32", max_obs=8, max_samples=B)
    with pytest.raises(binding.PlanError) as e:
        pl.step_resident([B])          # nothing uploaded
    assert e.value.status == binding.PLAN_ECAPACITY
    pl.upload([sc])
    with pytest.raises(binding.PlanError) as e:
        pl.step_resident([B + 1])      # too many samples
    assert e.value.status == binding.PLAN_ECAPACITY
    with pytest.raises(binding.PlanError) as e:
        pl.set_state(0, mu=[1.0, 2.0], sigma=[[-1.0, 0.0], [0.0, 1.0]])
    assert e.value.status == binding.PLAN_EINVAL
    pl.close()
