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
