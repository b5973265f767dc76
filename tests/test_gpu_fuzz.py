"""Seeded random configurations through plan_solve against the FP64 oracle:
basis width n in {8, 11, 16}, horizons m on both sides of the 128-step slot
boundary, 0 to 32 obstacles, 1, 2 or 4 set-point segments, with and without
goal entries, straight and curved roads, 1 to 40 samples (ragged against
every tile size), the plain FP64 path and the fused FP32 kernel at a random
shape.  Each case draws its own configuration from
its index, so a failure names a reproducible case."""
import numpy as np
import pytest
import torch

from oracle import lower
from oracle.basis import bernstein
from paper_2212_02224_gb300 import scenegen as sg

from gpu_common import compare, planner, to_dev

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1), (1, 2), (1, 4), (1, 5), (1, 7), (1, 8), (2, 1), (2, 2), (2, 4), (4, 1)]


def _case(idx):
    s = sg.Stream(9000 + idx)
    pick = lambda seq: seq[int(s.integers(0, len(seq) - 1, 1)[0])]
    n_coef = pick([8, 11, 16])
    m = pick([40, 77, 100, 128, 129, 150, 200])
    n_obs = pick([0, 1, 5, 12, 20, 32])
    n_seg = pick([1, 2, 4])
    goal = bool(s.integers(0, 1, 1)[0])
    road = bool(s.integers(0, 1, 1)[0])
    prec = pick(["fp64", "fp32", "fp32"])
    shape = pick(SHAPES)
    n_lanes = pick([2, 3, 4])
    B = pick([1, 7, 24, 33, 40])
    prm = sg.Params(m=m, n_coef=n_coef, n_seg=n_seg, goal=goal, inner_iters=40)
    sc = sg.make_scene(7000 + idx, n_lanes=n_lanes, n_obs=n_obs,
                       obs_x=(10.0, 10.0 + 0.8 * m))
    if road:
        kappa = float(s.uniform(0.005, 0.02, 1)[0])
        sc.road = sg.curved_road(n_lanes, kappa=kappa, bend=(20.0, 120.0),
                                 narrow_at=pick([None, 60.0]))
    p = sg.make_samples(8000 + idx, sc, B, n_seg,
                        goal_tf=(m - 1) * prm.dt if goal else None)
    return prm, sc, p, prec, shape


@pytest.mark.parametrize("idx", range(40))
def test_random_configuration_matches_oracle(idx):
    prm, sc, p, prec, shape = _case(idx)
    pl = planner(prm, prec, max_obs=max(sc.n_obs, 1), max_samples=len(p))
    if prec == "fp32":
        pl.set_tuning(*shape)
    xi, r, cu = pl.solve(sc, to_dev(p))
    torch.cuda.synchronize()
    out = xi.cpu().numpy(), r.cpu().numpy(), cu.cpu().numpy()
    pl.close()
    ref = lower.solve(p, sc, prm, bernstein(prm.m, prm.n_coef, prm.dt))
    compare(prec, prm, *out, *ref, sc=sc, p=p)
