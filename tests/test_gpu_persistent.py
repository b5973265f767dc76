"""The persistent form of the fused FP32 kernel (one wave of CTAs, samples taken
from a device counter) against the one-tile-per-CTA form: the same bits for
every shape, scene mix, road profile and goal entries, for batches that are
ragged against the sample groups; the counter is reset between launches of
different sizes; the graph-captured MPC cycle gives the same result; and one
batch is compared with the oracle directly."""
import numpy as np
import pytest
import torch

from oracle import lower
from oracle.basis import bernstein
from paper_2212_02224_gb300 import binding
from paper_2212_02224_gb300 import scenegen as sg

from gpu_common import compare, planner, to_dev

pytestmark = pytest.mark.gpu


def _host(out):
    torch.cuda.synchronize()
    return tuple(t.cpu().numpy() for t in out)


def _solve(prm, sc, p, mode, shape, max_obs=32):
    pl = planner(prm, "fp32", max_obs=max_obs, max_samples=len(p))
    pl.set_tuning(*shape)
    pl.set_persistent(mode)
    out = _host(pl.solve(sc, to_dev(p), want_status=True))
    pl.close()
    return out


def _same(a, b):
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("shape", [(1, 7), (1, 1), (1, 4), (1, 8),
                                   (2, 2), (4, 1)])   # the last two: one CTA per tile in either mode
@pytest.mark.parametrize("B", [1, 33, 1000])
def test_dense_traffic_forms_agree(shape, B):
    prm, sc, _ = sg.workload(1, inner_iters=40)
    p = sg.make_samples(71, sc, B, prm.n_seg)
    _same(_solve(prm, sc, p, "on", shape), _solve(prm, sc, p, "off", shape))


@pytest.mark.parametrize("shape", [(2, 2), (2, 4), (1, 4), (1, 8)])
def test_long_horizon_forms_agree(shape):
    # m = 200, n = 16, 30 obstacles: the eight-slot and two-warp instantiations
    prm, sc, _ = sg.workload(4, inner_iters=30)
    p = sg.make_samples(72, sc, 515, prm.n_seg)
    _same(_solve(prm, sc, p, "on", shape), _solve(prm, sc, p, "off", shape))


def test_goal_entries_forms_agree():
    prm, sc, _ = sg.workload(1, inner_iters=40, goal=True)
    p = sg.make_samples(73, sc, 301, prm.n_seg, goal_tf=(prm.m - 1) * prm.dt)
    for shape in [(1, 4), (1, 7)]:
        _same(_solve(prm, sc, p, "on", shape), _solve(prm, sc, p, "off", shape))


def _batch(seed=74, S=9, road=True):
    prm = sg.Params(m=100, n_coef=11, inner_iters=30)
    scenes, Bs = [], []
    rng = np.random.default_rng(seed)
    for i in range(S):
        sc = sg.make_scene(seed + i, n_lanes=3, n_obs=int(rng.integers(0, 21)))
        if road and i % 3 == 1:
            sc.road = sg.curved_road(3, kappa=0.01, bend=(20.0, 120.0))
        scenes.append(sc)
        Bs.append(int(rng.integers(1, 300)))
    p = np.concatenate([sg.make_samples(seed + 50 + i, scenes[i], Bs[i], prm.n_seg)
                        for i in range(S)])
    return prm, scenes, Bs, p


def _solve_batch(prm, scenes, Bs, p, mode, shape):
    pl = planner(prm, "fp32", max_obs=20, max_samples=sum(Bs), max_scenes=len(scenes))
    pl.set_tuning(*shape)
    pl.set_persistent(mode)
    out = _host(pl.solve_batch(scenes, Bs, to_dev(p), want_status=True))
    pl.close()
    return out


@pytest.mark.parametrize("shape", [(1, 4), (1, 8), (1, 1)])
def test_scene_mix_with_roads_forms_agree(shape):
    # each group restages its scene data whenever its next sample belongs to
    # another scene; scenes without obstacles and with road profiles are mixed
    prm, scenes, Bs, p = _batch()
    _same(_solve_batch(prm, scenes, Bs, p, "on", shape),
          _solve_batch(prm, scenes, Bs, p, "off", shape))


def test_counter_is_reset_between_launches():
    # one context, persistent launches of decreasing and increasing size on the
    # same stream: each must solve every one of its samples
    prm, sc, _ = sg.workload(1, inner_iters=20)
    sizes = [1000, 33, 1, 517, 1000]
    ps = [sg.make_samples(80 + i, sc, B, prm.n_seg) for i, B in enumerate(sizes)]
    ref = [_solve(prm, sc, p, "off", (1, 4)) for p in ps]
    pl = planner(prm, "fp32", max_obs=32, max_samples=1000)
    pl.set_tuning(1, 4)
    pl.set_persistent("on")
    for p, want in zip(ps, ref):
        got = _host(pl.solve(sc, to_dev(p), want_status=True))
        _same(got, want)
        assert (got[3] == binding.PLAN_OK).all()
    pl.close()


def test_graph_captured_cycle_forms_agree():
    prm, sc, B = sg.workload(1, inner_iters=30, outer_iters=3)
    res = {}
    for mode in ("on", "off"):
        pl = planner(prm, "fp32", max_obs=32, max_samples=B)
        pl.set_tuning(1, 4)
        pl.set_persistent(mode)
        pl.upload([sc])
        pl.set_state(0, seed=31, step=0)
        out = []
        for _ in range(2):
            pl.step_resident([B])
            out.append(pl.get_result(0))
        res[mode] = (out, pl.get_state(0))
        pl.close()
    assert res["on"][0] == res["off"][0]
    np.testing.assert_array_equal(res["on"][1]["mu"], res["off"][1]["mu"])
    np.testing.assert_array_equal(res["on"][1]["sigma"], res["off"][1]["sigma"])


def test_persistent_form_matches_the_oracle():
    prm, sc, _ = sg.workload(1, inner_iters=40)
    p = sg.make_samples(75, sc, 37, prm.n_seg)
    xi, r, cu, st = _solve(prm, sc, p, "on", (1, 4))
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    xi_o, r_o, cu_o = lower.solve(p, sc, prm, basis)
    compare("fp32", prm, xi, r, cu, xi_o, r_o, cu_o, sc=sc, p=p)
    assert (st == binding.PLAN_OK).all()


def test_invalid_mode_is_rejected():
    prm, _, _ = sg.workload(0)
    pl = planner(prm, "fp32", max_obs=8, max_samples=64)
    with pytest.raises(binding.PlanError) as e:
        pl.set_persistent(7)
    assert e.value.status == binding.PLAN_EINVAL
    pl.set_persistent("auto")
    pl.close()
