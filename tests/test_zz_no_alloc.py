"""The allocation-free float64 solve (plan_solve_fp64_noalloc) against the
context-based plan_solve on the float64 path.

The entry point serves callers that may not allocate device memory (a host
application that owns every allocation in a fixed pool, or a real-time loop
that must not enter an allocator after start-up).  Its scratch is a fixed
array inside the library, shared by every call, so this file checks two calls
in a row on the same stream.  It is named to be collected last, and it passes
both on its own in a fresh process and after the other tests."""
import numpy as np
import pytest
import torch

from paper_2212_02224_gb300 import binding, scenegen as sg

from gpu_common import FP64_XI_REL, planner, to_dev

pytestmark = pytest.mark.gpu


def _cmp(a, b, name):
    scale = max(1.0, float(np.abs(b).max()))
    err = float(np.abs(a - b).max()) / scale
    assert err <= FP64_XI_REL, f"{name}: relative error {err}"


def test_noalloc_matches_context_solve_twice():
    prm, sc, _ = sg.workload(1, inner_iters=40)
    B = 200
    cases = [sg.make_samples(900, sc, B, prm.n_seg), sg.make_samples(901, sc, B, prm.n_seg)]
    pl = planner(prm, "fp64", max_obs=16, max_samples=B)
    cfg = binding.make_config(prm, binding.PLAN_PREC_FP64, 16, B)
    stream = torch.cuda.current_stream().cuda_stream
    for p in cases:           # two calls in a row share the library's scratch array
        pt = to_dev(p)
        xi_ref, r_ref, cu_ref = pl.solve(sc, pt)
        xi = torch.full_like(xi_ref, float("nan"))
        r = torch.full_like(r_ref, float("nan"))
        cu = torch.full_like(cu_ref, float("nan"))
        binding.plan_solve_fp64_noalloc(cfg, sc, pt.data_ptr(), B, xi.data_ptr(), r.data_ptr(),
                                        cu.data_ptr(), stream)
        torch.cuda.synchronize()
        _cmp(xi.cpu().numpy(), xi_ref.cpu().numpy(), "xi")
        _cmp(r.cpu().numpy(), r_ref.cpu().numpy(), "resid")
        _cmp(cu.cpu().numpy(), cu_ref.cpu().numpy(), "cu")
    pl.close()


def _noalloc(cfg, sc, p, want_xi=True):
    B = p.shape[0]
    n = cfg.n_coef
    xi = torch.full((B, 2 * n), float("nan"), dtype=torch.float64, device="cuda")
    r = torch.full((B,), float("nan"), dtype=torch.float64, device="cuda")
    cu = torch.full((B,), float("nan"), dtype=torch.float64, device="cuda")
    binding.plan_solve_fp64_noalloc(cfg, sc, p.data_ptr(), B, xi.data_ptr() if want_xi else None,
                                    r.data_ptr(), cu.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
    return xi, r, cu


def test_noalloc_at_every_limit_then_a_smaller_call():
    """One call at all five limits at once (B = 256, m = 128, 32 obstacles,
    16 coefficients, 4 segments), so that every region of the scratch array is
    used to its end, then a smaller call (fewer obstacles, shorter horizon,
    narrower basis) on the same stream, which must not see the first call's
    leftovers.  Both against plan_solve on the float64 path."""
    big = sg.Params(m=128, n_coef=16, n_seg=4, inner_iters=15)
    sc_big = sg.make_scene(4321, n_lanes=5, n_obs=32, obs_x=(8.0, 140.0))
    p_big = sg.make_samples(11, sc_big, 256, 4)
    small, sc_small, _ = sg.workload(0, inner_iters=25, m=60)
    p_small = sg.make_samples(12, sc_small, 17, small.n_seg)
    for prm, sc, p in ((big, sc_big, p_big), (small, sc_small, p_small)):
        B = p.shape[0]
        cfg = binding.make_config(prm, binding.PLAN_PREC_FP64, sc.n_obs, B)
        pt = to_dev(p)
        xi, r, cu = _noalloc(cfg, sc, pt)
        pl = planner(prm, "fp64", max_obs=sc.n_obs, max_samples=B)
        xi_ref, r_ref, cu_ref = pl.solve(sc, pt)
        torch.cuda.synchronize()
        pl.close()
        _cmp(xi.cpu().numpy(), xi_ref.cpu().numpy(), "xi")
        _cmp(r.cpu().numpy(), r_ref.cpu().numpy(), "resid")
        _cmp(cu.cpu().numpy(), cu_ref.cpu().numpy(), "cu")


def test_noalloc_matches_the_oracle():
    """A small case straight against the FP64 CPU oracle (1e-6 relative)."""
    from oracle import lower
    from oracle.basis import bernstein
    prm, sc, _ = sg.workload(0, inner_iters=30)
    p = sg.make_samples(13, sc, 24, prm.n_seg)
    cfg = binding.make_config(prm, binding.PLAN_PREC_FP64, sc.n_obs, 24)
    xi, r, cu = _noalloc(cfg, sc, to_dev(p))
    torch.cuda.synchronize()
    xo, ro, co = lower.solve(p, sc, prm, bernstein(prm.m, prm.n_coef, prm.dt))
    scale = np.maximum(1.0, np.abs(xo).max(axis=1))
    assert (np.abs(xi.cpu().numpy() - xo).max(axis=1) / scale).max() <= FP64_XI_REL
    assert (np.abs(r.cpu().numpy() - ro) / np.maximum(1.0, np.abs(ro))).max() <= FP64_XI_REL
    assert (np.abs(cu.cpu().numpy() - co) / np.maximum(1.0, np.abs(co))).max() <= FP64_XI_REL


def test_noalloc_with_goal_entries():
    """The goal rows of Eq. final_boundary on the allocation-free path."""
    prm, sc, _ = sg.workload(1, inner_iters=30, goal=True, n_seg=2)
    p = sg.make_samples(14, sc, 64, prm.n_seg, goal_tf=(prm.m - 1) * prm.dt)
    cfg = binding.make_config(prm, binding.PLAN_PREC_FP64, sc.n_obs, 64)
    pt = to_dev(p)
    xi, r, cu = _noalloc(cfg, sc, pt)
    pl = planner(prm, "fp64", max_obs=sc.n_obs, max_samples=64)
    xi_ref, r_ref, cu_ref = pl.solve(sc, pt)
    torch.cuda.synchronize()
    pl.close()
    _cmp(xi.cpu().numpy(), xi_ref.cpu().numpy(), "xi")
    _cmp(r.cpu().numpy(), r_ref.cpu().numpy(), "resid")


def test_noalloc_rejects_sizes_beyond_its_limits():
    prm, sc, _ = sg.workload(1, inner_iters=5)
    cfg = binding.make_config(prm, binding.PLAN_PREC_FP64, 16, 512)
    p = to_dev(sg.make_samples(3, sc, 257, prm.n_seg))
    out = torch.empty(257, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.PlanError) as e:
        binding.plan_solve_fp64_noalloc(cfg, sc, p.data_ptr(), 257, None, out.data_ptr(),
                                        out.data_ptr())
    assert e.value.status == binding.PLAN_ECAPACITY
    assert "256" in str(e.value)
