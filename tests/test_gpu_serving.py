"""The serving loop (continuous batching of MPC cycles) and MPC episodes.

* A request's result is the same alone and in a mix of other scenes admitted
  into the same waves (the kernel shape is fixed per executor and every
  sample, selection and update is per scene, so the equality is exact).
* An episode of several cycles through the server (warm starts kept in the
  device table, scenes advanced with plan_advance) matches the same episode
  through plan_step, and on the FP64 path matches the oracle's episode.
* Many requests of mixed horizons and sizes all complete; the loop batches
  them into fewer waves than requests.
"""
import numpy as np
import pytest
import torch

from oracle import mpc
from paper_2212_02224_gb300 import binding, scenegen as sg
from paper_2212_02224_gb300.planner import Planner, Server, advance


pytestmark = pytest.mark.gpu


def _prm(**kw):
    prm, _, _ = sg.workload(1, inner_iters=25, outer_iters=2, n_elite_c=60, n_elite=20)
    for k, v in kw.items():
        setattr(prm, k, v)
    return prm


def _scene(i, n_obs=None):
    s = sg.Stream(900 + i)
    n = int(s.integers(4, 16, 1)[0]) if n_obs is None else n_obs
    return sg.make_scene(1000 + i, n_lanes=4, n_obs=n)


def test_result_same_alone_and_in_the_mix():
    prm = _prm()
    target = _scene(0)
    srv = Server(prm, max_obs=24, max_samples=4096, max_scenes=16, max_executors=2)
    t = srv.submit(target, 300, episode=77, seed=5)
    alone = srv.wait(t)
    srv.close()

    srv = Server(prm, max_obs=24, max_samples=4096, max_scenes=16, max_executors=1)
    rng = np.random.default_rng(3)
    scenes = [_scene(i) for i in range(1, 12)]      # made up front: submissions come in a burst
    sizes = [int(rng.integers(100, 600)) for _ in scenes]
    tickets = []
    for i, (sc, b) in enumerate(zip(scenes, sizes), start=1):
        tickets.append(srv.submit(sc, b, episode=i, seed=i))
        if i == 6:
            tt = srv.submit(target, 300, episode=77, seed=5)
    mixed = srv.wait(tt)
    others = [srv.wait(x) for x in tickets]
    info = srv.info()
    srv.close()
    assert all(np.isfinite(o["cost"]) for o in others)
    assert info["waves"] < 12           # requests shared waves
    for key in ("p", "xi", "cost", "resid", "cu", "index"):
        assert mixed[key] == alone[key], key


def test_server_episode_matches_plan_step():
    """Three cycles through the server vs three plan_step calls with the
    distribution carried by the caller: the same bits (plan_step factors the
    carried covariance on the device, as the server's selection did)."""
    prm = _prm()
    sc0 = _scene(21, n_obs=10)
    srv = Server(prm, max_obs=16, max_samples=2048, max_scenes=4, max_executors=1)
    pl = Planner(prm, prec="fp32", max_obs=16, max_samples=2048)
    pl.set_tuning(1, 4)                       # the executors' fixed shape
    sc_s, sc_p = sc0, sc0
    mu = sigma = None
    for c in range(3):
        r_s = srv.wait(srv.submit(sc_s, 400, episode=5, seed=11))
        r_p = pl.step(sc_p, 400, mu=mu, sigma=sigma, seed=11, step=c)
        mu, sigma = r_p["mu"], r_p["sigma"]
        for key in ("p", "xi", "cost", "resid", "cu", "index"):
            assert r_s[key] == r_p[key], (c, key)
        sc_s = advance(prm, sc_s, r_s["xi"])
        sc_p = advance(prm, sc_p, r_p["xi"])
    srv.close()
    pl.close()


@pytest.mark.parametrize("outer", [2, 4])
def test_fresh_cycle_through_the_server_matches_plan_step_bits(outer):
    """plan_step's captured graph draws the normals of outer iterations 2..L on
    a side stream beside the previous solve; the server's waves draw them inside
    the sampling kernel.  A fresh cycle (nothing carried through the host) gives
    the same bits on both."""
    prm = _prm(outer_iters=outer)
    sc = _scene(23, n_obs=8)
    srv = Server(prm, max_obs=16, max_samples=2048, max_scenes=4, max_executors=1)
    pl = Planner(prm, prec="fp32", max_obs=16, max_samples=2048)
    pl.set_tuning(1, 4)                       # the executors' fixed shape
    r_s = srv.wait(srv.submit(sc, 400, episode=7, seed=13))
    r_p = pl.step(sc, 400, seed=13, step=0)
    srv.close()
    pl.close()
    for key in ("p", "xi", "cost", "resid", "cu", "index"):
        assert r_s[key] == r_p[key], key


def test_fp64_episode_matches_oracle_episode():
    """Receding horizon on the FP64 path (plan_step + plan_advance) against the
    oracle's episode (upper.plan with warm starts + mpc.advance)."""
    prm, sc, B = sg.workload(0, inner_iters=20, outer_iters=2)
    ref, _ = mpc.episode(sc, prm, 3, B, seed=9)
    pl = Planner(prm, prec="fp64", max_obs=8, max_samples=B)
    cur = sc
    mu = sigma = None
    for c in range(3):
        r = pl.step(cur, B, mu=mu, sigma=sigma, seed=9, step=c)
        assert r["index"] == ref[c]["best"]
        np.testing.assert_allclose(r["xi"], ref[c]["xi"], rtol=1e-6, atol=1e-6)
        np.testing.assert_allclose(r["mu"], ref[c]["mu"], rtol=1e-6, atol=1e-6)
        mu, sigma = r["mu"], r["sigma"]
        cur = advance(prm, cur, r["xi"])
    pl.close()


def test_mixed_horizons_and_sizes_complete():
    prm = _prm()
    srv = Server(prm, max_obs=24, max_samples=6000, max_scenes=24, max_executors=4)
    rng = np.random.default_rng(8)
    reqs = [(_scene(100 + i), int(rng.integers(64, 900)), int(rng.choice([80, 100, 120])))
            for i in range(40)]
    tickets = [srv.submit(sc, b, m=m, episode=1000 + i, seed=i) for i, (sc, b, m) in enumerate(reqs)]
    res = [srv.wait(t) for t in tickets]
    info = srv.info()
    srv.close()
    assert all(np.isfinite(r["cost"]) and r["latency_us"] > 0 for r in res)
    assert info["completed"] == 40 and info["waves"] < 40 and info["executors"] >= 3


def test_server_errors():
    prm = _prm()
    srv = Server(prm, max_obs=4, max_samples=512, max_scenes=4, max_executors=1, max_episodes=2)
    with pytest.raises(binding.PlanError) as e:
        srv.submit(_scene(1, n_obs=8), 100, episode=1)
    assert e.value.status == binding.PLAN_ECAPACITY
    with pytest.raises(binding.PlanError) as e:
        srv.submit(_scene(1, n_obs=2), 513, episode=1)
    assert e.value.status == binding.PLAN_ECAPACITY
    srv.wait(srv.submit(_scene(1, n_obs=2), 100, episode=1))
    srv.wait(srv.submit(_scene(2, n_obs=2), 100, episode=2))
    with pytest.raises(binding.PlanError) as e:
        srv.submit(_scene(3, n_obs=2), 100, episode=3)      # episode table full
    assert e.value.status == binding.PLAN_ECAPACITY
    srv.end_episode(1)
    srv.wait(srv.submit(_scene(3, n_obs=2), 100, episode=3))
    with pytest.raises(binding.PlanError) as e:
        binding.plan_poll(srv.srv, 123456, 0)                # unknown ticket
    assert e.value.status == binding.PLAN_EINVAL
    srv.close()


def test_poll_any_returns_every_ticket_once():
    """plan_poll_any hands out completed tickets in completion order; tickets
    already taken by plan_poll are skipped; results equal those of plan_poll."""
    prm = _prm()
    srv = Server(prm, max_obs=24, max_samples=4096, max_scenes=8, max_executors=2)
    scenes = [_scene(20 + i) for i in range(9)]
    tickets = [srv.submit(sc, 200 + 37 * i, episode=300 + i, seed=i) for i, sc in enumerate(scenes)]
    direct = srv.wait(tickets[4])                  # one ticket taken by plan_poll
    got = {}
    while len(got) < len(tickets) - 1:
        r = srv.poll_any(2_000_000)
        assert r is not None, "no completion within 2 s"
        t, res = r
        assert t not in got and t != tickets[4]
        got[t] = res
    assert set(got) == set(tickets) - {tickets[4]}
    assert srv.poll_any(0) is None                 # nothing left
    srv.close()
    assert all(np.isfinite(v["cost"]) for v in got.values()) and np.isfinite(direct["cost"])
    # the same requests through plan_poll give the same results
    srv = Server(prm, max_obs=24, max_samples=4096, max_scenes=8, max_executors=2)
    again = [srv.submit(sc, 200 + 37 * i, episode=300 + i, seed=i) for i, sc in enumerate(scenes)]
    for t0, t1 in zip(tickets, again):
        r1 = srv.wait(t1)
        r0 = direct if t0 == tickets[4] else got[t0]
        assert r1["index"] == r0["index"] and r1["cost"] == r0["cost"]
    srv.close()
