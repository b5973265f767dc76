"""Shared helpers of the GPU parity tests (no method arithmetic here)."""
import numpy as np
import torch

from oracle.basis import bernstein
from paper_2212_02224_gb300 import scenegen as sg
from paper_2212_02224_gb300.planner import Planner

# Tolerances.  FP64 path: coefficients within 1e-6 relative to max(1, |xi|inf)
# of the oracle.  FP32 path: every trajectory position within 1e-3 m (the
# Euclidean distance between the GPU's and the oracle's point at each t), the
# constraint residual within 1e-3 and the driving cost within 1e-4 relative.
FP64_XI_REL = 1e-6
FP32_POS_M = 1e-3
FP32_RESID = 1e-3
FP32_COST_REL = 1e-4


def planner(prm, prec, max_obs=32, max_samples=4096, max_scenes=1):
    return Planner(prm, prec=prec, max_obs=max_obs, max_samples=max_samples, max_scenes=max_scenes)


def to_dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def positions(xi, prm):
    W = bernstein(prm.m, prm.n_coef, prm.dt)[0]
    n = prm.n_coef
    return xi[:, :n] @ W.T, xi[:, n:] @ W.T


def position_error(xi_a, xi_b, prm):
    """Largest Euclidean distance between the two plans' points over all t."""
    xa, ya = positions(np.atleast_2d(xi_a), prm)
    xb, yb = positions(np.atleast_2d(xi_b), prm)
    return float(np.hypot(xa - xb, ya - yb).max())


def compare(prec, prm, xi_g, r_g, cu_g, xi_o, r_o, cu_o):
    """Assert parity of one batch; returns the error summary."""
    if prec == "fp64":
        scale = np.maximum(1.0, np.abs(xi_o).max(axis=1))
        e_xi = (np.abs(xi_g - xi_o).max(axis=1) / scale).max()
        e_r = (np.abs(r_g - r_o) / np.maximum(1.0, np.abs(r_o))).max()
        e_cu = (np.abs(cu_g - cu_o) / np.maximum(1.0, np.abs(cu_o))).max()
        assert e_xi <= FP64_XI_REL, f"xi rel err {e_xi}"
        assert e_r <= FP64_XI_REL and e_cu <= FP64_XI_REL, (e_r, e_cu)
        return dict(xi=e_xi, r=e_r, cu=e_cu)
    e_pos = position_error(xi_g, xi_o, prm)
    e_r = np.abs(r_g - r_o).max()
    e_cu = (np.abs(cu_g - cu_o) / np.maximum(1e-12, np.abs(cu_o))).max()
    assert e_pos <= FP32_POS_M, f"position err {e_pos} m"
    assert e_r <= FP32_RESID, f"resid err {e_r}"
    assert e_cu <= FP32_COST_REL, f"cost rel err {e_cu}"
    return dict(pos=e_pos, r=e_r, cu=e_cu)


def scene_with(seed, n_lanes, n_obs, **kw):
    return sg.make_scene(seed, n_lanes=n_lanes, n_obs=n_obs, **kw)
