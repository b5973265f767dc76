"""A second, independent statement of Alg. 2 that pins the parts of
``oracle.lower.project`` that no invariant fixes: the multiplier step of
Eq. (update_lagrange), whose printed factor is rho/2, and which iterate the
road curvature is taken at in the velocity clip of Eq. (clip_d_v), which the
paper prints as kappa(^k xi) (the previous iterate, while the angles come
from ^{k+1} xi; the analysis of step split_xy says the same).

Nothing here reuses the oracle's assembly or solvers.  It works one sample
at a time, one constraint row at a time, in plain Python floats:

* the Bernstein basis from its definition (math.comb), with derivatives by
  the difference identity;
* the rows of F (each obstacle's position rows, then the velocity and the
  acceleration rows, per axis) and of G (upper and lower lane rows on the y
  block) as explicit coefficient vectors with their targets;
* the alpha/d step with math.atan2 / cos / sin per (t, obstacle);
* the road curvature and lane limits by walking the knot list;
* the xi-step of Eq. (split_xy) by the null-space method: a particular
  solution of A xi = b plus the minimiser over null(A) of the augmented
  Lagrangian, whose Hessian is summed row by row (the oracle uses a KKT LU
  solve instead);
* the multiplier update as the per-row sum
  lambda -= rho/2 sum_r f_r (f_r . xi - h_r) + rho/2 sum_r g_r (g_r . xi - e_r + s_r).

The scene is built so that both readings matter within two iterations: a
road whose curvature grows linearly from 0 to 0.1 1/m over the first 50 m
(so kappa at ^0 xi and at ^1 xi differ wherever the iterates' positions
differ, and the centripetal bound of the velocity clip, sqrt(c_max / kappa),
is below the planned speed over most of the horizon), a lateral set-point
beyond the upper lane limit (the Step-1 trajectory violates the lane rows at
its last timesteps), and an obstacle on the way.
"""
import math

import numpy as np
import pytest
from scipy.linalg import null_space

from oracle import lower
from oracle.basis import bernstein
from paper_2212_02224_gb300 import scenegen as sg


# --------------------------------------------------------------------------- tiny scene

def _setup():
    prm = sg.Params(m=16, n_coef=6, n_seg=1, inner_iters=2, dt=0.2)
    road = np.array([[0.0, 0.0, 0.0, 7.0],
                     [50.0, 0.1, 0.0, 7.0]])
    sc = sg.Scene(ego=np.array([0.0, 1.75, 16.0, 0.0, 0.0, 0.0]), n_lanes=2, lane_width=3.5,
                  kappa_road=0.0,
                  obstacles=np.array([[14.0, 2.3, 6.0, 0.0, 2.8, 1.5]]), road=road)
    p = np.array([[9.0, 20.0]])          # y_d beyond y_ub = 6, v_d = 20 m/s
    return prm, sc, p


# --------------------------------------------------------------------------- restatement

def _basis_rows(m, n, dt):
    """W[t], Wd[t], Wdd[t] as lists of lists, from the Bernstein definition."""
    deg = n - 1
    tf = (m - 1) * dt

    def b(d, k, tau):
        if k < 0 or k > d:
            return 0.0
        return math.comb(d, k) * tau ** k * (1.0 - tau) ** (d - k)

    W, Wd, Wdd = [], [], []
    for t in range(m):
        tau = t / (m - 1)
        W.append([b(deg, k, tau) for k in range(n)])
        Wd.append([deg * (b(deg - 1, k - 1, tau) - b(deg - 1, k, tau)) / tf for k in range(n)])
        Wdd.append([deg * (deg - 1) * (b(deg - 2, k - 2, tau) - 2.0 * b(deg - 2, k - 1, tau)
                                       + b(deg - 2, k, tau)) / tf ** 2 for k in range(n)])
    return W, Wd, Wdd


def _dot(u, v):
    return sum(a * b for a, b in zip(u, v))


def _road(knots, margin, x):
    """kappa, y_lb, y_ub at arc length x: linear between knots, constant beyond."""
    if x <= knots[0][0]:
        k = knots[0]
        return k[1], k[2] + margin, k[3] - margin
    for a, b in zip(knots[:-1], knots[1:]):
        if x <= b[0]:
            w = (x - a[0]) / (b[0] - a[0])
            return (a[1] + w * (b[1] - a[1]), a[2] + w * (b[2] - a[2]) + margin,
                    a[3] + w * (b[3] - a[3]) - margin)
    k = knots[-1]
    return k[1], k[2] + margin, k[3] - margin


def _angle(sy, cx):
    return 0.0 if (sy == 0.0 and cx == 0.0) else math.atan2(sy, cx)


class _Sample:
    """One sample's Alg. 2 state, row by row."""

    def __init__(self, xi_bar, sc, prm, goal=None):
        self.prm, self.sc = prm, sc
        self.m, self.n = prm.m, prm.n_coef
        self.W, self.Wd, self.Wdd = _basis_rows(self.m, self.n, prm.dt)
        self.knots = [list(r) for r in np.asarray(sc.road)]
        self.xi_bar = [float(v) for v in xi_bar]
        self.obs = [list(map(float, o)) for o in np.asarray(sc.obstacles).reshape(-1, 6)]
        n = self.n
        # equality rows of Eq. (boundary_cond_initial): x block then y block
        self.A, self.b = [], []
        for axis in (0, 1):
            for mat, comp in ((self.W, 0), (self.Wd, 2), (self.Wdd, 4)):
                row = [0.0] * (2 * n)
                row[axis * n:(axis + 1) * n] = mat[0]
                self.A.append(row)
                self.b.append(float(sc.ego[axis + comp]))
        if goal is not None:
            # Eq. final_boundary: x(t_f) = x_f, y(t_f) = y_f, ydot(t_f) = 0
            x_f, y_f = goal
            for axis, mat, val in ((0, self.W, x_f), (1, self.W, y_f), (1, self.Wd, 0.0)):
                self.A.append(self._row(axis, mat[self.m - 1]))
                self.b.append(float(val))

    def _row(self, axis, basis_row, sign=1.0):
        r = [0.0] * (2 * self.n)
        r[axis * self.n:(axis + 1) * self.n] = [sign * v for v in basis_row]
        return r

    def state(self, xi, t):
        n = self.n
        cx, cy = xi[:n], xi[n:]
        return (_dot(self.W[t], cx), _dot(self.W[t], cy), _dot(self.Wd[t], cx),
                _dot(self.Wd[t], cy), _dot(self.Wdd[t], cx), _dot(self.Wdd[t], cy))

    def f_rows(self, xi, da_prev, x_kappa):
        """Rows (f_r, h_r) of F xi = h after Eqs. split_alpha_o and the clips;
        the curvature of the velocity clip is taken at positions x_kappa[t].
        Returns the rows and the new d_a."""
        prm = self.prm
        rows, da_new = [], []
        st = [self.state(xi, t) for t in range(self.m)]
        for axis in (0, 1):
            for (x0, y0, vxo, vyo, a, b) in self.obs:
                for t in range(self.m):
                    tt = t * prm.dt
                    xo, yo = x0 + vxo * tt, y0 + vyo * tt
                    dx, dy = st[t][0] - xo, st[t][1] - yo
                    al = _angle(dy / b, dx / a)
                    d = max(1.0, math.hypot(dx / a, dy / b))
                    h = xo + a * d * math.cos(al) if axis == 0 else yo + b * d * math.sin(al)
                    rows.append((self._row(axis, self.W[t]), h))
        hv, ha = [], []
        for t in range(self.m):
            x, y, vx, vy, ax, ay = st[t]
            al_v, al_a = _angle(vy, vx), _angle(ay, ax)
            S = abs(math.sin(al_a - al_v))
            kap = abs(_road(self.knots, prm.lane_margin, x_kappa[t])[0])
            vmin_b = max(prm.v_min, math.sqrt(da_prev[t] * S / prm.kappa_max))
            c2 = math.cos(al_v) ** 2
            vmax_b = prm.v_max if kap * c2 == 0.0 else min(prm.v_max, math.sqrt(prm.c_max / (kap * c2)))
            dv = min(max(math.hypot(vx, vy), vmin_b), vmax_b)
            kd = dv * dv * prm.kappa_max
            amax_b = prm.a_max if S * prm.a_max <= kd else kd / S
            dacc = min(max(math.hypot(ax, ay), 0.0), amax_b)
            da_new.append(dacc)
            hv.append((dv * math.cos(al_v), dv * math.sin(al_v)))
            ha.append((dacc * math.cos(al_a), dacc * math.sin(al_a)))
        for axis in (0, 1):
            for t in range(self.m):
                rows.append((self._row(axis, self.Wd[t]), hv[t][axis]))
            for t in range(self.m):
                rows.append((self._row(axis, self.Wdd[t]), ha[t][axis]))
        return rows, da_new

    def g_rows(self, xi):
        """Lane rows (g_r, e_r) at the positions of xi: y <= y_ub(x), -y <= -y_lb(x)."""
        out = []
        for t in range(self.m):
            x = self.state(xi, t)[0]
            _, ylb, yub = _road(self.knots, self.prm.lane_margin, x)
            out.append((self._row(1, self.W[t]), yub))
        for t in range(self.m):
            x = self.state(xi, t)[0]
            _, ylb, yub = _road(self.knots, self.prm.lane_margin, x)
            out.append((self._row(1, self.W[t], -1.0), -ylb))
        return out

    def xi_step(self, lam, frows, grows, slack):
        """Eq. (split_xy) by the null-space method."""
        rho = self.prm.rho
        nn = 2 * self.n
        H = np.eye(nn)
        c = np.array(self.xi_bar) + np.array(lam)
        for f, h in frows:
            fv = np.array(f)
            H += rho * np.outer(fv, fv)
            c += rho * h * fv
        for (g, e), s in zip(grows, slack):
            gv = np.array(g)
            H += rho * np.outer(gv, gv)
            c += rho * (e - s) * gv
        A, b = np.array(self.A), np.array(self.b)
        xp = np.linalg.lstsq(A, b, rcond=None)[0]
        Z = null_space(A)
        z = np.linalg.solve(Z.T @ H @ Z, Z.T @ (c - H @ xp))
        return list(xp + Z @ z)

    def run(self, iters, step_factor=0.5, kappa_lag=True):
        """Alg. 2 for `iters` iterations.  The defaults are the paper's
        readings (multiplier step rho/2, curvature at ^k xi); the others exist
        only to show that this scene tells the readings apart."""
        prm = self.prm
        xi = list(self.xi_bar)
        lam = [0.0] * (2 * self.n)
        st = [self.state(xi, t) for t in range(self.m)]
        da = [min(math.hypot(s[4], s[5]), prm.a_max) for s in st]
        x_k = [s[0] for s in st]
        frows, da = self.f_rows(xi, da, x_k)                     # alpha^0, d^0 at xi^0
        grows = self.g_rows(xi)                                  # e(^0 xi)
        slack = [max(0.0, e - _dot(g, xi)) for g, e in grows]    # s^0
        for _ in range(iters):
            x_k = [self.state(xi, t)[0] for t in range(self.m)]  # positions of ^k xi
            xi = self.xi_step(lam, frows, grows, slack)          # split_xy with e(^k xi)
            x_new = [self.state(xi, t)[0] for t in range(self.m)]
            frows, da = self.f_rows(xi, da, x_k if kappa_lag else x_new)  # clips; kappa(^k xi)
            grows = self.g_rows(xi)                              # e(^{k+1} xi)
            slack = [max(0.0, e - _dot(g, xi)) for g, e in grows]  # update_slack
            step = step_factor * prm.rho                         # update_lagrange: rho/2 as printed
            for f, h in frows:
                r = _dot(f, xi) - h
                lam = [l - step * fv * r for l, fv in zip(lam, f)]
            for (g, e), s in zip(grows, slack):
                r = _dot(g, xi) - e + s
                lam = [l - step * gv * r for l, gv in zip(lam, g)]
        return np.array(xi)


# --------------------------------------------------------------------------- pins

@pytest.mark.parametrize("iters", [1, 2, 3])
def test_project_matches_rowwise_restatement(iters):
    """lower.project equals the row-by-row statement of Alg. 2 to 1e-9 (relative
    to the coefficients' size) after 1, 2 and 3 iterations."""
    prm, sc, p = _setup()
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    xb = lower.step1(p, sc, prm, basis)
    got = lower.project(xb, sc, prm, basis, iters=iters)[0]
    want = _Sample(xb[0], sc, prm).run(iters)
    scale = max(1.0, float(np.max(np.abs(want))))
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-9 * scale)


def test_scene_exercises_both_readings():
    """The scene tells both readings apart within two iterations: with a
    multiplier step of rho (instead of rho/2), or with the curvature taken at
    the current iterate (instead of ^k xi), the restatement's xi^2 moves by far
    more than the comparison tolerance above.  This guards the pin against a
    scene in which neither reading matters."""
    prm, sc, p = _setup()
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    xb = lower.step1(p, sc, prm, basis)[0]
    ref = _Sample(xb, sc, prm).run(2)
    scale = max(1.0, float(np.max(np.abs(ref))))
    alt_step = _Sample(xb, sc, prm).run(2, step_factor=1.0)
    alt_kappa = _Sample(xb, sc, prm).run(2, kappa_lag=False)
    assert np.max(np.abs(alt_step - ref)) > 1e-6 * scale
    assert np.max(np.abs(alt_kappa - ref)) > 1e-6 * scale
