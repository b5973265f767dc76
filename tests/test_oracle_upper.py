"""Pins of the oracle's Alg. 1 pieces: Philox4x32-10 against its published
known-answer vectors, Box-Muller moments, selections against Python's sort,
the distribution update against hand-made elites with known moments, and the
whole loop against brute force on a tiny scene."""
import os

import numpy as np
import pytest

from oracle import lower, upper
from oracle.basis import bernstein
from paper_2212_02224_gb300 import scenegen as sg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(x, 16) for x in line.split()]
            rows.append((v[:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat())
def test_philox_known_answers(ctr, key, out):
    got = upper.philox4x32_10(np.array([ctr], dtype=np.uint64), key)[0]
    assert [int(v) for v in got] == out


def test_uniform_and_normal_moments():
    u = upper.uniforms(upper.raw_words(50000, 4, 3, 123, 9))
    assert u.min() > 0 and u.max() < 1
    assert abs(u.mean() - 0.5) < 0.005 and abs(u.var() - 1 / 12) < 0.002
    z = upper.normals(50000, 8, 2, 77, 0)
    assert abs(z.mean()) < 0.01
    np.testing.assert_allclose(np.cov(z.T), np.eye(8), atol=0.02)
    # distinct outer iterations and steps give distinct streams
    z2 = upper.normals(1000, 8, 3, 77, 0)
    z3 = upper.normals(1000, 8, 2, 77, 1)
    assert not np.allclose(z[:1000], z2) and not np.allclose(z[:1000], z3)


def test_gaussian_draw_moments():
    prm = sg.Params(n_seg=2)
    mu = np.array([1.0, -2.0, 10.0, 20.0])
    A = np.array([[1.0, 0, 0, 0], [0.5, 2.0, 0, 0], [0, 0.3, 1.5, 0], [0.2, 0, 0.1, 3.0]])
    sigma = A @ A.T
    p = upper.draw_gaussian(200000, mu, sigma, prm, 2, 5, 0)
    np.testing.assert_allclose(p.mean(0), mu, atol=0.03)
    np.testing.assert_allclose(np.cov(p.T), sigma + 1e-6 * np.eye(4), rtol=0.03, atol=0.03)


def test_initial_draws_and_moments():
    prm = sg.Params(n_seg=2)
    sc = sg.make_scene(1, n_lanes=4, n_obs=0)
    p = upper.draw_initial(100000, sc, prm, 3, 0)
    assert set(np.unique(p[:, :2])) == set(sc.lane_centres())
    assert p[:, 2:].min() >= prm.v_des_lo and p[:, 2:].max() <= prm.v_des_hi
    mu, sigma = upper.initial_moments(sc, prm)
    np.testing.assert_allclose(p.mean(0), mu, rtol=0.01)
    np.testing.assert_allclose(np.cov(p.T), sigma, rtol=0.02, atol=0.4)


def test_select_lowest_matches_sorted_with_ties():
    rng = np.random.default_rng(0)
    keys = rng.integers(0, 20, size=300).astype(float)   # many ties
    got = upper.select_lowest(keys, 40)
    want = [i for _, i in sorted((k, i) for i, k in enumerate(keys))][:40]
    assert list(got) == want
    among = rng.choice(300, 90, replace=False)
    got = upper.select_lowest(keys, 25, among=among)
    want = [i for _, i in sorted((keys[i], i) for i in among)][:25]
    assert list(got) == want


def test_update_distribution_equal_weights():
    """Equal costs give equal s_j: the update blends in the plain elite mean and
    the elite scatter around the new mean."""
    prm = sg.Params(eta=0.6)
    mu = np.array([1.0, 2.0])
    sigma = np.diag([4.0, 9.0])
    pe = np.array([[0.0, 0.0], [2.0, 0.0], [0.0, 2.0], [2.0, 2.0]])
    mu1, s1 = upper.update_distribution(mu, sigma, pe, np.full(4, 3.0), prm)
    np.testing.assert_allclose(mu1, 0.4 * mu + 0.6 * np.array([1.0, 1.0]))
    dev = pe - mu1
    np.testing.assert_allclose(s1, 0.4 * sigma + 0.6 * (dev.T @ dev) / 4)


def test_update_distribution_weights_follow_costs():
    """Two elites whose costs differ by gamma*ln(3): weights 3:1."""
    prm = sg.Params(eta=1.0, gamma=0.9)
    pe = np.array([[0.0], [4.0]])
    cost = np.array([10.0, 10.0 + 0.9 * np.log(3.0)])
    mu1, s1 = upper.update_distribution(np.zeros(1), np.eye(1), pe, cost, prm)
    np.testing.assert_allclose(mu1, [1.0])
    np.testing.assert_allclose(s1, [[0.75 * 1.0 + 0.25 * 9.0]])


def test_plan_matches_brute_force_on_tiny_scene():
    """Alg. 1 finds a behaviour at least as good as a 1-D grid search over v_d
    (within one grid step's worth of cost), for a single-lane road."""
    prm = sg.Params(m=30, n_coef=8, inner_iters=15, outer_iters=4, n_elite_c=24,
                    n_elite=8, v_des_lo=5.0, v_des_hi=30.0)
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    sc = sg.make_scene(4, n_lanes=1, n_obs=1, obs_x=(25.0, 25.0), obs_vx=(12.0, 12.0))
    sc.ego[2] = 15.0
    grid = np.linspace(5.0, 30.0, 101)
    pg = np.stack([np.full_like(grid, sc.lane_centres()[0]), grid], axis=1)
    _, r, cu = lower.solve(pg, sc, prm, basis)
    best_grid = (cu + r).min()
    step_cost = np.abs(np.diff(cu + r)).max()
    out = upper.plan(sc, prm, 64, seed=5, basis=basis)
    assert out["cost"] <= best_grid + step_cost
    # the returned pair is consistent with a direct solve of the returned p
    xs, r1, cu1 = lower.solve(out["p"][None], sc, prm, basis)
    np.testing.assert_allclose(xs[0], out["xi"], rtol=1e-12, atol=1e-10)
    np.testing.assert_allclose(cu1[0] + r1[0], out["cost"], rtol=1e-12)


def test_plan_cost_trend_non_increasing():
    """Sec. V-B: the best elite cost saturates over the outer iterations."""
    prm, sc, B = sg.workload(0, inner_iters=20, outer_iters=5)
    out = upper.plan(sc, prm, B, seed=3, keep_trace=True)
    best = [float((t["cu"] + t["r"])[t["E"][0]]) for t in out["trace"]]
    assert best[-1] <= best[0]
