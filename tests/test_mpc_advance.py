"""plan_advance (host code of the library) against the oracle's receding-horizon
step, and the oracle's step against a closed form."""
import numpy as np
import pytest

from oracle import mpc
from oracle.basis import bernstein
from paper_2212_02224_gb300 import binding, build, scenegen as sg
import os


def _lib():
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    return binding.load()


def test_oracle_advance_closed_form():
    """Cruise at 17 m/s on a lane centre: after 5 steps the ego is still at
    17 m/s, the frame shifts by 17 * 0.25 m and obstacles move accordingly."""
    prm = sg.Params()
    sc = sg.make_scene(3, n_lanes=2, n_obs=2)
    n = prm.n_coef
    tf = (prm.m - 1) * prm.dt
    k = np.arange(n) / (n - 1)
    xi = np.concatenate([17.0 * tf * k, np.full(n, 1.75)])
    nxt = mpc.advance(sc, xi, prm, 5)
    np.testing.assert_allclose(nxt.ego, [0.0, 1.75, 17.0, 0.0, 0.0, 0.0], atol=1e-9)
    t = 5 * prm.dt
    np.testing.assert_allclose(nxt.obstacles[:, 0], sc.obstacles[:, 0] + sc.obstacles[:, 2] * t - 17.0 * t)


@pytest.mark.parametrize("n_coef,m,steps", [(11, 100, 5), (16, 200, 5), (8, 37, 3), (11, 100, 0)])
def test_plan_advance_matches_oracle(n_coef, m, steps):
    _lib()
    prm = sg.Params(m=m, n_coef=n_coef)
    sc = sg.make_scene(7, n_lanes=3, n_obs=4)
    rng = np.random.default_rng(1)
    xi = np.concatenate([np.linspace(0, 90, n_coef) + rng.normal(0, 1, n_coef),
                         5.0 + rng.normal(0, 0.5, n_coef)])
    cfg = binding.make_config(prm, binding.PLAN_PREC_FP64, 8, 8)
    got = binding.plan_advance(cfg, sc, xi, steps)
    want = mpc.advance(sc, xi, prm, steps, bernstein(m, n_coef, prm.dt))
    np.testing.assert_allclose(got.ego, want.ego, rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(np.array(got.obstacles), want.obstacles, rtol=1e-12, atol=1e-10)
    assert got.n_lanes == sc.n_lanes and got.lane_width == sc.lane_width


def test_plan_advance_rejects_bad_steps():
    _lib()
    prm = sg.Params()
    sc = sg.make_scene(7, n_lanes=3, n_obs=0)
    cfg = binding.make_config(prm, binding.PLAN_PREC_FP64, 8, 8)
    with pytest.raises(binding.PlanError):
        binding.plan_advance(cfg, sc, np.zeros(2 * prm.n_coef), prm.m)
