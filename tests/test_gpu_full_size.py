"""Parity at the full sizes of the multi-scene and scale workloads, in the
launch configuration the benchmarks use, on sampled outputs that the oracle
solves one by one:

* 256 scenes, N ~ U{4..20}, B ~ U{256..2048} (288 454 samples) in one
  batched FP32 solve at the batched benchmark's shape (1 warp per sample,
  2 samples per CTA);
* one scene with 30 obstacles on 6 lanes, m = 200, n = 16, B = 32 768, FP32
  solve at the autotuned shape of the scale benchmark's largest point.

Each sampled result meets the FP32 bar (positions within 1e-3 m, residual
within 1e-3, cost within 1e-4 relative)."""
import numpy as np
import pytest
import torch

from oracle import lower
from oracle.basis import bernstein
from paper_2212_02224_gb300 import scenegen as sg

from gpu_common import compare, planner, to_dev

pytestmark = pytest.mark.gpu


def test_batched_workload_full_size_sampled():
    prm, scenes, Bs = sg.batched_workload(S=256)
    ps = [sg.make_samples(9 + i, scenes[i], Bs[i], prm.n_seg) for i in range(len(scenes))]
    total = sum(Bs)
    pl = planner(prm, "fp32", max_obs=20, max_samples=total, max_scenes=len(scenes))
    pl.set_tuning(1, 2)                  # the batched benchmark's shape
    xi, r, cu = pl.solve_batch(scenes, Bs, to_dev(np.concatenate(ps)))
    torch.cuda.synchronize()
    xi, r, cu = xi.cpu().numpy(), r.cpu().numpy(), cu.cpu().numpy()
    pl.close()
    assert np.isfinite(r).all() and np.isfinite(cu).all()
    offs = np.concatenate([[0], np.cumsum(Bs)])
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    pick = sg.Stream(31)
    for sidx in np.unique(pick.integers(0, len(scenes) - 1, 8)):
        js = np.unique(pick.integers(0, Bs[sidx] - 1, 3))
        xo, ro, co = lower.solve(ps[sidx][js], scenes[sidx], prm, basis)
        g = offs[sidx] + js
        compare("fp32", prm, xi[g], r[g], cu[g], xo, ro, co, sc=scenes[sidx], p=ps[sidx][js])


def test_scale_workload_largest_point_sampled():
    prm, sc, B = sg.workload(4, B=32768)
    p = sg.make_samples(303, sc, B, prm.n_seg)
    pl = planner(prm, "fp32", max_obs=32, max_samples=B)
    pl.autotune(sc, B)
    xi, r, cu = pl.solve(sc, to_dev(p))
    torch.cuda.synchronize()
    xi, r, cu = xi.cpu().numpy(), r.cpu().numpy(), cu.cpu().numpy()
    pl.close()
    assert np.isfinite(r).all() and np.isfinite(cu).all()
    idx = np.unique(sg.Stream(41).integers(0, B - 1, 16))
    xo, ro, co = lower.solve(p[idx], sc, prm, bernstein(prm.m, prm.n_coef, prm.dt))
    compare("fp32", prm, xi[idx], r[idx], cu[idx], xo, ro, co, sc=sc, p=p[idx])
