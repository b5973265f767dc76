"""Alg. 1 (bi-level optimisation) around the FP64 lower level, batched.

Sampling (Alg. 1 line 4), ConstraintEliteSet / EliteSet (lines 10-13), the
distribution update of Eqs. (mean_update, cov_update, s_formula) and the
returned best pair (Alg. 1 last line).

Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC'11), written here from that definition, and
Box-Muller in float64.  Counter = (j, l | c << 16, step_lo, step_hi) and key =
(seed_lo, seed_hi) for sample j, outer iteration l (1-based), 4-word block c
and MPC episode step; entry e of p_j uses word e % 4 of block e // 4.

Readings adopted (the paper leaves these open):
  * first iteration of a fresh episode draws y_d uniformly over lane centres
    and v_d ~ U[v_des_lo, v_des_hi] per segment; with goal entries, x_f =
    x0 + v t_f with v ~ U[v_des_lo, v_des_hi] (t_f = (m - 1) dt, x0 the ego
    position) and y_f uniformly over lane centres.  mu^0 / Sigma^0 are the
    moments of that distribution.  Later iterations, and the first iteration
    of a warm-started cycle, draw N(mu, Sigma + cov_eps I).
  * ties in both selections go to the lower sample index.
  * s_j is computed with the minimum elite cost subtracted before exp
    (identical after normalisation; avoids underflow at gamma = 0.9).
  * learning rate eta and the covariance jitter are parameters (0.9, 1e-6).
"""
from __future__ import annotations

import math

import numpy as np

from . import lower

_M0 = 0xD2511F53
_M1 = 0xCD9E8D57
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_U32 = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds.  ctr: (..., 4) uint32-valued array, key: (2,)
    ints.  Returns (..., 4) uint64 array holding the 32-bit outputs."""
    c = [np.asarray(ctr[..., i], dtype=np.uint64) for i in range(4)]
    k0, k1 = np.uint64(key[0] & _U32), np.uint64(key[1] & _U32)
    m0, m1 = np.uint64(_M0), np.uint64(_M1)
    mask = np.uint64(_U32)
    s32 = np.uint64(32)
    for rnd in range(10):
        if rnd:
            k0 = np.uint64((int(k0) + _W0) & _U32)
            k1 = np.uint64((int(k1) + _W1) & _U32)
        p0 = m0 * c[0]
        p1 = m1 * c[2]
        hi0, lo0 = p0 >> s32, p0 & mask
        hi1, lo1 = p1 >> s32, p1 & mask
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return np.stack(c, axis=-1)


def raw_words(B: int, d_p: int, l: int, seed: int, step: int):
    """uint32 words (B, d_p) for outer iteration l of MPC step `step`."""
    nblk = (d_p + 3) // 4
    out = np.empty((B, 4 * nblk), dtype=np.uint64)
    j = np.arange(B, dtype=np.uint64)
    key = (seed & _U32, (seed >> 32) & _U32)
    for c in range(nblk):
        ctr = np.stack([j, np.full(B, (l | (c << 16)) & _U32, dtype=np.uint64),
                        np.full(B, step & _U32, dtype=np.uint64),
                        np.full(B, (step >> 32) & _U32, dtype=np.uint64)], axis=1)
        out[:, 4 * c:4 * c + 4] = philox4x32_10(ctr, key)
    return out


def uniforms(words):
    """(x + 0.5) * 2^-32, in (0, 1)."""
    return (words.astype(np.float64) + 0.5) * 2.0 ** -32


def normals(B: int, d_p: int, l: int, seed: int, step: int):
    """Standard normals (B, d_p) by Box-Muller on word pairs (2q, 2q+1)."""
    u = uniforms(raw_words(B, d_p, l, seed, step))
    r = np.sqrt(-2.0 * np.log(u[:, 0::2]))
    th = 2.0 * math.pi * u[:, 1::2]
    z = np.empty_like(u)
    z[:, 0::2] = r * np.cos(th)
    z[:, 1::2] = r * np.sin(th)
    return z[:, :d_p]


def initial_moments(scene, prm):
    """mu^0, Sigma^0 of the first-iteration uniform distribution."""
    ns = prm.n_seg
    L, w = scene.n_lanes, scene.lane_width
    lane_mu, lane_var = L * w / 2.0, w * w * (L * L - 1) / 12.0
    v_mu, v_var = 0.5 * (prm.v_des_lo + prm.v_des_hi), (prm.v_des_hi - prm.v_des_lo) ** 2 / 12.0
    mu = [lane_mu] * ns + [v_mu] * ns
    var = [lane_var] * ns + [v_var] * ns
    if getattr(prm, "goal", False):
        tf = (prm.m - 1) * prm.dt
        mu += [float(scene.ego[0]) + tf * v_mu, lane_mu]
        var += [tf * tf * v_var, lane_var]
    return np.array(mu), np.diag(var)


def draw_initial(B, scene, prm, seed, step):
    """First iteration of a fresh episode: lane-centre y_d, uniform v_d (and,
    with goal entries, x_f = x0 + U[v_des_lo, v_des_hi] t_f, lane-centre y_f)."""
    ns = prm.n_seg
    goal = getattr(prm, "goal", False)
    d_p = 2 * ns + (2 if goal else 0)
    u = uniforms(raw_words(B, d_p, 1, seed, step))[:, :d_p]
    centres = (np.arange(scene.n_lanes) + 0.5) * scene.lane_width

    def lane(uu):
        return centres[np.minimum(np.floor(uu * scene.n_lanes).astype(np.int64), scene.n_lanes - 1)]

    def speed(uu):
        return prm.v_des_lo + (prm.v_des_hi - prm.v_des_lo) * uu

    p = np.empty((B, d_p))
    p[:, :ns] = lane(u[:, :ns])
    p[:, ns:2 * ns] = speed(u[:, ns:2 * ns])
    if goal:
        p[:, 2 * ns] = float(scene.ego[0]) + (prm.m - 1) * prm.dt * speed(u[:, 2 * ns])
        p[:, 2 * ns + 1] = lane(u[:, 2 * ns + 1])
    return p


def draw_gaussian(B, mu, sigma, prm, l, seed, step):
    """Alg. 1 line 4: p_j ~ N(mu, Sigma), via the Cholesky factor of Sigma + eps I."""
    d_p = mu.shape[0]
    Lc = np.linalg.cholesky(sigma + prm.cov_eps * np.eye(d_p))
    return mu[None, :] + normals(B, d_p, l, seed, step) @ Lc.T


def select_lowest(keys, count, among=None):
    """Indices of the `count` lowest keys, ascending, ties to the lower index."""
    idx = np.arange(len(keys)) if among is None else np.asarray(among)
    k = np.asarray(keys)[idx]
    order = np.lexsort((idx, k))
    return idx[order[:count]]


def update_distribution(mu, sigma, p_elite, cost_elite, prm):
    """Eqs. (mean_update, cov_update, s_formula)."""
    s = np.exp(-(cost_elite - cost_elite.min()) / prm.gamma)
    S = s.sum()
    mu_new = (1.0 - prm.eta) * mu + prm.eta * (s[:, None] * p_elite).sum(axis=0) / S
    dev = p_elite - mu_new[None, :]
    cov = (s[:, None, None] * dev[:, :, None] * dev[:, None, :]).sum(axis=0) / S
    sigma_new = (1.0 - prm.eta) * sigma + prm.eta * cov
    return mu_new, sigma_new


def plan(scene, prm, B, seed, step=0, mu=None, sigma=None, basis=None, iters=None,
         keep_trace=False):
    """Alg. 1.  Returns dict(p, xi, cost, r, cu, mu, sigma[, trace]) where
    p, xi are the best pair of the final EliteSet.  A fresh episode is one with
    mu=None; otherwise (mu, sigma) warm-start the first iteration."""
    from .basis import bernstein
    if basis is None:
        basis = bernstein(prm.m, prm.n_coef, prm.dt)
    fresh = mu is None
    if fresh:
        mu, sigma = initial_moments(scene, prm)
    nc = prm.n_elite_c if prm.n_elite_c > 0 else min(B, 3 * prm.n_elite)
    trace = []
    for l in range(1, prm.outer_iters + 1):
        if l == 1 and fresh:
            p = draw_initial(B, scene, prm, seed, step)
        else:
            p = draw_gaussian(B, mu, sigma, prm, l, seed, step)
        xs, r, cu = lower.solve(p, scene, prm, basis, iters)
        C = select_lowest(r, min(nc, B))
        cost = cu + r
        E = select_lowest(cost, min(prm.n_elite, len(C)), among=C)
        mu, sigma = update_distribution(mu, sigma, p[E], cost[E], prm)
        best = E[0]
        if keep_trace:
            trace.append(dict(p=p, r=r, cu=cu, C=C, E=E, mu=mu.copy(), sigma=sigma.copy()))
    out = dict(p=p[best], xi=xs[best], cost=float(cost[best]), r=float(r[best]),
               cu=float(cu[best]), mu=mu, sigma=sigma, best=int(best))
    if keep_trace:
        out["trace"] = trace
    return out
