"""Per-sample status of plan_solve / plan_solve_batch: a sample whose input is
not finite is flagged PLAN_ENONFINITE, only that sample, and every other
sample keeps its parity with the oracle."""
import numpy as np
import pytest
import torch

from oracle import lower
from oracle.basis import bernstein
from paper_2212_02224_gb300 import binding, scenegen as sg

from gpu_common import compare, planner, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3"])
@pytest.mark.parametrize("bad", ["nan_setpoint", "inf_velocity"])
def test_nonfinite_sample_is_flagged_alone(prec, bad):
    prm, sc, _ = sg.workload(1, inner_iters=40)
    p = sg.make_samples(77, sc, 40, prm.n_seg)
    j_bad = 13
    p[j_bad, 0 if bad == "nan_setpoint" else 1] = np.nan if bad == "nan_setpoint" else np.inf
    pl = planner(prm, prec, max_obs=sc.n_obs, max_samples=len(p))
    xi, r, cu, st = pl.solve(sc, to_dev(p), want_status=True)
    torch.cuda.synchronize()
    xi, r, cu, st = xi.cpu().numpy(), r.cpu().numpy(), cu.cpu().numpy(), st.cpu().numpy()
    pl.close()
    assert st[j_bad] == binding.PLAN_ENONFINITE
    ok = np.arange(len(p)) != j_bad
    assert (st[ok] == binding.PLAN_OK).all()
    xo, ro, co = lower.solve(p[ok], sc, prm, bernstein(prm.m, prm.n_coef, prm.dt))
    compare("fp32" if prec == "tf32x3" else prec, prm, xi[ok], r[ok], cu[ok], xo, ro, co, sc=sc,
            p=p[ok])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_status_in_a_batch_of_scenes(prec):
    prm, scenes, Bs = sg.batched_workload(S=3, seed=41, B_range=(10, 40), N_range=(2, 8),
                                          inner_iters=20)
    tot = sum(Bs)
    p = np.concatenate([sg.make_samples(50 + i, scenes[i], Bs[i], prm.n_seg) for i in range(3)])
    bad = [Bs[0] + 2, tot - 1]           # one in the second scene, the very last sample
    p[bad[0], 1] = np.nan
    p[bad[1], 0] = -np.inf
    pl = planner(prm, prec, max_obs=16, max_samples=tot, max_scenes=3)
    _, _, _, st = pl.solve_batch(scenes, Bs, to_dev(p), want_status=True)
    torch.cuda.synchronize()
    st = st.cpu().numpy()
    pl.close()
    want = np.full(tot, binding.PLAN_OK)
    want[bad] = binding.PLAN_ENONFINITE
    np.testing.assert_array_equal(st, want)


def test_status_without_xi_output():
    """The status also covers the solution when xi is not written out."""
    prm, sc, _ = sg.workload(0, inner_iters=10)
    p = sg.make_samples(3, sc, 20, prm.n_seg)
    p[5, 1] = np.nan
    pl = planner(prm, "fp32", max_obs=sc.n_obs, max_samples=20)
    _, r, cu, st = pl.solve(sc, to_dev(p), want_xi=False, want_status=True)
    st = st.cpu().numpy()
    pl.close()
    assert st[5] == binding.PLAN_ENONFINITE and (np.delete(st, 5) == binding.PLAN_OK).all()
