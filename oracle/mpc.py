"""Receding-horizon use of Alg. 1 (Sec. V-A, MPC-Bi-Level), FP64 oracle.

Test infrastructure only (see the package docstring).  After each planning
cycle the ego executes the first `steps` elements of the plan; the next cycle
starts from the trajectory state at t_steps, with the neighbours advanced at
constant velocity, in a frame shifted so that the ego is again at x = 0, and
warm-starts the sampling distribution with the cycle's final (mu, Sigma).
"""
from __future__ import annotations

import copy

import numpy as np

from . import lower, upper
from .basis import bernstein


def advance(scene, xi, prm, steps: int = 5, basis=None):
    """Next scene after executing `steps` elements of plan xi (2n coefficients)."""
    if basis is None:
        basis = bernstein(prm.m, prm.n_coef, prm.dt)
    x, y, xd, yd, xdd, ydd = (v[0, steps] for v in lower.kinematics(np.atleast_2d(xi), basis))
    t = steps * prm.dt
    nxt = copy.deepcopy(scene)
    nxt.ego = np.array([0.0, y, xd, yd, xdd, ydd])
    ob = np.array(scene.obstacles, dtype=np.float64).reshape(-1, 6).copy()
    ob[:, 0] = ob[:, 0] + ob[:, 2] * t - x
    ob[:, 1] = ob[:, 1] + ob[:, 3] * t
    nxt.obstacles = ob
    nxt.road_origin = float(getattr(scene, "road_origin", 0.0)) + x   # frame moves with the ego
    return nxt


def episode(scene, prm, cycles: int, B: int, seed: int, steps: int = 5, basis=None):
    """`cycles` MPC cycles; returns the list of per-cycle plan() outputs and scenes."""
    if basis is None:
        basis = bernstein(prm.m, prm.n_coef, prm.dt)
    out, scenes = [], [scene]
    mu = sigma = None
    for c in range(cycles):
        res = upper.plan(scenes[-1], prm, B, seed, step=c, mu=mu, sigma=sigma, basis=basis)
        out.append(res)
        mu, sigma = res["mu"], res["sigma"]
        scenes.append(advance(scenes[-1], res["xi"], prm, steps, basis))
    return out, scenes
