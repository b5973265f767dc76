"""Tensor-core modes of the lower-level solve (tcgen05 contractions) through the
C ABI against the FP64 oracle.

TF32X3 splits every operand into a TF32 head and tail and is held to the
FP32 bar (positions within 1e-3 m, residual within 1e-3, cost within 1e-4
relative).  TF32 and BF16 round every operand once.  Their bars are derived
for each case from the operand-rounding error model (tests/error_model.py):
three times the largest deviation the model predicts for the same scene,
samples and K (unit roundoff 2^-11 and 2^-8), never below the FP32 bar."""
import numpy as np
import pytest
import torch

from oracle import lower, upper
from oracle.basis import bernstein
from paper_2212_02224_gb300 import binding, scenegen as sg

import error_model
from gpu_common import (FP32_COST_REL, FP32_POS_M, FP32_RESID, compare, planner, positions,
                        scene_with, to_dev)

pytestmark = pytest.mark.gpu

FP32_BARS = (FP32_POS_M, FP32_RESID, FP32_COST_REL)
MODES = ["tf32x3", "tf32", "bf16"]


def _oracle(prm, sc, p):
    return lower.solve(p, sc, prm, bernstein(prm.m, prm.n_coef, prm.dt))


def _run(prec, prm, sc, p, max_obs=32):
    pl = planner(prm, prec, max_obs=max_obs, max_samples=max(len(p), 1))
    xi, r, cu = pl.solve(sc, to_dev(p))
    torch.cuda.synchronize()
    out = xi.cpu().numpy(), r.cpu().numpy(), cu.cpu().numpy()
    pl.close()
    return out


def _check(prec, prm, g, o, sc, p):
    """Parity within the mode's bars: the FP32 bar for TF32X3, the bars derived
    from the operand-rounding model for TF32 and BF16."""
    if prec == "tf32x3":
        compare("fp32", prm, *g, *o, sc=sc, p=p)
        return
    bp, br, bc = error_model.derived_bars(prm, sc, p, prec, FP32_BARS)
    xg, yg = positions(g[0], prm)
    xo, yo = positions(o[0], prm)
    e_pos = float(np.hypot(xg - xo, yg - yo).max())
    e_r = np.abs(g[1] - o[1])
    e_cu = (np.abs(g[2] - o[2]) / np.maximum(1e-12, np.abs(o[2]))).max()
    assert e_pos <= bp, f"{prec}: position err {e_pos} m"
    assert (e_r <= br).all(), f"{prec}: resid err {e_r.max()}"
    assert e_cu <= bc, f"{prec}: cost rel err {e_cu}"


@pytest.mark.parametrize("prec", MODES)
def test_small_plain_workload(prec):
    prm, sc, B = sg.workload(0)
    p = sg.make_samples(101, sc, B, prm.n_seg)
    _check(prec, prm, _run(prec, prm, sc, p), _oracle(prm, sc, p), sc, p)


@pytest.mark.parametrize("prec", MODES)
def test_dense_traffic_scene(prec):
    prm, sc, _ = sg.workload(1)
    p = sg.make_samples(202, sc, 96, prm.n_seg)
    _check(prec, prm, _run(prec, prm, sc, p), _oracle(prm, sc, p), sc, p)


@pytest.mark.parametrize("prec", MODES)
def test_dense_traffic_full_batch_sampled(prec):
    """B = 1000 (125 CTAs of 8 samples); TF32X3 compares every sample with the
    oracle, TF32 and BF16 (whose bars need the error model's runs) 96 sampled."""
    prm, sc, B = sg.workload(1)
    p = sg.make_samples(303, sc, B, prm.n_seg)
    xi, r, cu = _run(prec, prm, sc, p)
    idx = np.arange(B) if prec == "tf32x3" else np.unique(sg.Stream(7).integers(0, B - 1, 96))
    _check(prec, prm, (xi[idx], r[idx], cu[idx]), _oracle(prm, sc, p[idx]), sc, p[idx])


@pytest.mark.parametrize("prec", MODES)
@pytest.mark.parametrize("case", ["no_obstacles", "single_sample", "four_segments",
                                  "ragged_horizon", "wide_basis", "ragged_tile"])
def test_edge_cases(prec, case):
    if case == "no_obstacles":
        prm, sc, _ = sg.workload(0, inner_iters=30)
        sc.obstacles = np.zeros((0, 6))
        p = sg.make_samples(1, sc, 40, prm.n_seg)
    elif case == "single_sample":
        prm, sc, _ = sg.workload(1, inner_iters=40)
        p = sg.make_samples(2, sc, 1, prm.n_seg)
    elif case == "four_segments":
        prm, sc, _ = sg.workload(1, inner_iters=40, n_seg=4)
        p = sg.make_samples(3, sc, 50, 4)
    elif case == "ragged_horizon":
        prm = sg.Params(m=37, n_coef=8, inner_iters=30)
        sc = scene_with(4, 3, 5, obs_x=(5.0, 30.0))
        p = sg.make_samples(4, sc, 33, 1)
    elif case == "wide_basis":
        # degree-15 basis, 30 obstacles, the longest horizon of these modes
        prm = sg.Params(m=128, n_coef=16, inner_iters=40)
        sc = scene_with(5, 6, 30, obs_x=(10.0, 120.0))
        p = sg.make_samples(5, sc, 20, prm.n_seg)
    else:
        prm, sc, _ = sg.workload(1, inner_iters=50)
        p = sg.make_samples(6, sc, 61, prm.n_seg)      # 7 full tiles and one of 5
    _check(prec, prm, _run(prec, prm, sc, p, max_obs=max(sc.n_obs, 1)), _oracle(prm, sc, p), sc, p)


@pytest.mark.parametrize("prec", MODES)
def test_batched_scenes_uneven(prec):
    prm, scenes, Bs = sg.batched_workload(S=5, seed=77, B_range=(1, 40), N_range=(0, 14),
                                          inner_iters=40)
    ps = [sg.make_samples(500 + i, scenes[i], Bs[i], prm.n_seg) for i in range(5)]
    pl = planner(prm, prec, max_obs=20, max_samples=sum(Bs), max_scenes=5)
    xi, r, cu = pl.solve_batch(scenes, Bs, to_dev(np.concatenate(ps)))
    torch.cuda.synchronize()
    xi, r, cu = xi.cpu().numpy(), r.cpu().numpy(), cu.cpu().numpy()
    pl.close()
    off = 0
    for i in range(5):
        sl = slice(off, off + Bs[i])
        _check(prec, prm, (xi[sl], r[sl], cu[sl]), _oracle(prm, scenes[i], ps[i]), scenes[i], ps[i])
        off += Bs[i]


def test_mpc_cycle_tf32x3():
    """A whole Alg. 1 cycle in TF32X3: the returned pair is a valid lower-level
    solution of its own p (checked by the oracle), its cost close to the
    oracle's cycle."""
    prm, sc, B = sg.workload(0, inner_iters=30, outer_iters=3)
    pl = planner(prm, "tf32x3", max_obs=8, max_samples=B)
    res = pl.step(sc, B, seed=21, step=0)
    pl.close()
    ref = upper.plan(sc, prm, B, seed=21)
    xo, ro, co = _oracle(prm, sc, np.array([res["p"]]))
    xg, yg = positions(np.array([res["xi"]]), prm)
    xr, yr = positions(xo, prm)
    assert float(np.hypot(xg - xr, yg - yr).max()) <= FP32_POS_M
    assert abs(res["cost"] - (co[0] + ro[0])) <= 1e-4 * abs(co[0] + ro[0]) + 1e-3
    assert res["cost"] <= ref["cost"] * 1.05 + 1e-3


def test_repeat_is_bitwise_deterministic():
    prm, sc, _ = sg.workload(1, inner_iters=30)
    p = sg.make_samples(9, sc, 40, prm.n_seg)
    a = _run("tf32x3", prm, sc, p)
    b = _run("tf32x3", prm, sc, p)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


def test_bounded_wait_gives_up_and_the_device_stays_usable():
    """The tensor-core solve's mbarrier wait, run on a barrier that nothing
    arrives at, gives up after its bound and reports PLAN_ETIMEOUT through the
    error flag; the device then still runs a tensor-core solve to parity."""
    assert binding.plan_probe_wait_timeout(0) == binding.PLAN_EINVAL
    for _ in range(2):
        assert binding.plan_probe_wait_timeout(2000) == binding.PLAN_ETIMEOUT
    prm, sc, B = sg.workload(0, inner_iters=20)
    p = sg.make_samples(303, sc, 40, prm.n_seg)
    _check("tf32x3", prm, _run("tf32x3", prm, sc, p), _oracle(prm, sc, p), sc, p)
