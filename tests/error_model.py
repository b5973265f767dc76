"""Error model of the reduced-precision contraction modes (test infrastructure).

The tensor-core modes round the operands of the two contractions of every
Alg. 2 iteration -- the forward evaluation W delta of Eq. param and the
transposed contraction of the residual rows onto the coefficients (Eq.
split_xy) -- to a narrower format and accumulate in float32.  This module
predicts what that does to the solution by propagating the standard model of
floating-point rounding, fl(x) = x (1 + e) with |e| <= u (Higham, "Accuracy
and Stability of Numerical Algorithms", 2nd ed., Sec. 2.2), through the
method itself: the FP64 oracle runs Alg. 2 while every contraction operand
carries a rounding error of that model, and the model's prediction is how
far the result moves from the unperturbed oracle.

Where the rounding enters, as in the kernels (increment form on
delta = xi - xi_bar):
  * forward: x(t) = x_ref(t) + sum_k W[t,k] delta_k with W[t,k] rounded once
    (the same error e_W[t,k] at every iteration) and delta_k rounded afresh
    at every iteration (e_d,k);
  * transposed: each residual row R = h - F xi is rounded afresh at every
    iteration (e_R) and its basis row once (e_WT); a row is exactly zero where
    its projection is inactive (the clip leaves the point where it is), so
    inactive rows carry no error.
The errors e are drawn uniformly from [-u, u]; u is the unit roundoff of the
operand format: TF32 (10 stored mantissa bits) 2^-11, BF16 (7 bits) 2^-8, and
the split-TF32 head-plus-tail representation about 2^-21.

This is a first-order model: it leaves out the float32 arithmetic of the
projections and of the xi-step, which is why the modes are also never held
to less than the float32 bar.  The oracle module itself is not modified:
the perturbation wraps two of its functions for the duration of one call.
"""
from __future__ import annotations

import numpy as np

from oracle import lower
from oracle.basis import bernstein

UNIT_ROUNDOFF = {"tf32": 2.0 ** -11, "bf16": 2.0 ** -8, "tf32x3": 2.0 ** -21}


def predicted_deviation(prm, sc, p, u, draws: int = 3, seed: int = 0, iters=None, with_ref=False):
    """Per sample, the largest deviation over `draws` realisations of the
    rounding model with unit roundoff u: (position error [m], the Euclidean
    distance at the worst t; |r - r_ref|; |c_u - c_u,ref| / |c_u,ref|), and
    the unperturbed r_ref as a fourth entry when with_ref."""
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    W = basis[0]
    n, m, N = prm.n_coef, prm.m, sc.n_obs
    p = np.atleast_2d(np.asarray(p, dtype=np.float64))
    xb = lower.step1(p, sc, prm, basis)
    ref = lower.project(xb, sc, prm, basis, iters, p=p)
    r_ref, cu_ref = lower.score(ref, sc, prm, basis)
    kin0, ad0 = lower.kinematics, lower.alpha_d_step
    d_pos = np.zeros(len(p))
    d_r = np.zeros(len(p))
    d_cu = np.zeros(len(p))
    for d in range(draws):
        rng = np.random.default_rng(seed + d)
        e_w = [rng.uniform(-u, u, (m, n)) for _ in range(3)]     # rounding of W, Wd, Wdd
        state = {"e_wt": None, "last": None}

        def kin(xi, basis_):
            out = kin0(xi, basis_)
            if xi.shape != xb.shape:
                return out
            dl = xi - xb
            e_d = rng.uniform(-u, u, dl.shape)                   # rounding of delta
            pert = []
            for q, v in enumerate(out):
                mat = basis_[q // 2]
                cols = slice((q % 2) * n, (q % 2 + 1) * n)
                pert.append(v + dl[:, cols] @ (mat * e_w[q // 2]).T
                            + (dl[:, cols] * e_d[:, cols]) @ mat.T)
            state["last"] = (out, tuple(pert))
            return tuple(pert)

        def rows(k):
            x, y, xd, yd, xdd, ydd = k
            return np.concatenate([np.tile(x, (1, N)), xd, xdd, np.tile(y, (1, N)), yd, ydd], axis=1)

        def alpha_d(xi, scene, prm_, basis_, da_prev, x_prev=None):
            h, da, parts = ad0(xi, scene, prm_, basis_, da_prev, x_prev)
            exact, pert = state["last"]
            R = rows(pert) - h                                   # the residual the kernel forms
            active = np.abs(R) > 1e-9 * (1.0 + np.abs(h))
            if state["e_wt"] is None:
                state["e_wt"] = rng.uniform(-u, u, R.shape[1])
            R = np.where(active, R * (1.0 + rng.uniform(-u, u, R.shape) + state["e_wt"][None, :]), 0.0)
            return rows(exact) - R, da, parts

        lower.kinematics, lower.alpha_d_step = kin, alpha_d
        try:
            xs = lower.project(xb, sc, prm, basis, iters, p=p)
            # the kernels score the final iterate from the same rounded forward
            # contraction, so the scoring sees the perturbed kinematics too
            r, cu = lower.score(xs, sc, prm, basis)
        finally:
            lower.kinematics, lower.alpha_d_step = kin0, ad0
        dx = xs[:, :n] @ W.T - ref[:, :n] @ W.T
        dy = xs[:, n:] @ W.T - ref[:, n:] @ W.T
        d_pos = np.maximum(d_pos, np.hypot(dx, dy).max(axis=1))
        d_r = np.maximum(d_r, np.abs(r - r_ref))
        d_cu = np.maximum(d_cu, np.abs(cu - cu_ref) / np.maximum(1e-12, np.abs(cu_ref)))
    return (d_pos, d_r, d_cu, r_ref) if with_ref else (d_pos, d_r, d_cu)


SAFETY = 3.0


def derived_bars(prm, sc, p, mode, floor, draws: int = 3, iters=None):
    """(position m, residual, relative cost) bars of a reduced-precision mode:
    SAFETY times the model's worst sample, never below `floor` (the float32
    bar, which covers the float32 arithmetic the model leaves out).  The
    residual bar is per sample (an array): the larger of that and 1e-4 |r|,
    as for the float32 path."""
    d_pos, d_r, d_cu, r_ref = predicted_deviation(prm, sc, p, UNIT_ROUNDOFF[mode], draws=draws,
                                                  iters=iters, with_ref=True)
    r_bar = np.maximum(max(floor[1], SAFETY * float(d_r.max())), 1e-4 * np.abs(r_ref))
    return (max(floor[0], SAFETY * float(d_pos.max())), r_bar,
            max(floor[2], SAFETY * float(d_cu.max())))
