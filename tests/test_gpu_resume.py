"""Checkpoint and resume of an episode through plan_get_state / plan_set_state:
an episode of four warm-started MPC cycles, interrupted after two (state
exported, context destroyed, a new context created and the state imported),
ends where the uninterrupted episode ends, bit for bit (the imported
covariance is factored on the device by the selection kernels' routine)."""
import numpy as np
import pytest

from paper_2212_02224_gb300 import scenegen as sg

from gpu_common import planner

pytestmark = pytest.mark.gpu


def _cycles(pl, sc, B, n):
    out = []
    for _ in range(n):
        pl.step_resident([B])
        out.append(pl.get_result(0))
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_resumed_episode_matches_uninterrupted(prec):
    prm, sc, B = sg.workload(0, inner_iters=30, outer_iters=3)
    pl = planner(prm, prec, max_obs=max(sc.n_obs, 1), max_samples=B)
    pl.upload([sc])
    pl.set_state(0, seed=21, step=0)
    whole = _cycles(pl, sc, B, 4)
    final_state = pl.get_state(0)
    pl.close()

    pl = planner(prm, prec, max_obs=max(sc.n_obs, 1), max_samples=B)
    pl.upload([sc])
    pl.set_state(0, seed=21, step=0)
    first = _cycles(pl, sc, B, 2)
    saved = pl.get_state(0)
    pl.close()
    assert saved["fresh"] == 0 and saved["step"] == 2

    pl = planner(prm, prec, max_obs=max(sc.n_obs, 1), max_samples=B)
    pl.upload([sc])
    pl.set_state(0, mu=saved["mu"], sigma=saved["sigma"], seed=saved["seed"], step=saved["step"],
                 fresh=saved["fresh"])
    second = _cycles(pl, sc, B, 2)
    resumed_state = pl.get_state(0)
    pl.close()

    assert first == whole[:2]                      # the same program up to the checkpoint
    assert second == whole[2:]                     # and after it, bit for bit
    assert resumed_state["step"] == final_state["step"] == 4
    np.testing.assert_array_equal(resumed_state["mu"], final_state["mu"])
    np.testing.assert_array_equal(resumed_state["sigma"], final_state["sigma"])
