"""Pins of the oracle's lower level: Step 1 (Alg. 1 line 7), the pieces of
Alg. 2 and the scoring, against closed forms, optimality conditions of the
paper's objectives written out term by term, constraint-set invariants, an
independent QP solve of the convex special case, and brute-force identities.
"""
import numpy as np
import pytest
from scipy.linalg import null_space
from scipy.optimize import minimize

from oracle import lower
from oracle.basis import bernstein
from paper_2212_02224_gb300 import scenegen as sg


def _prm(**kw):
    p = sg.Params(m=60, n_coef=11, inner_iters=30)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _scene(n_obs=3, seed=5, n_lanes=3, **kw):
    return sg.make_scene(seed, n_lanes=n_lanes, n_obs=n_obs, **kw)


# --------------------------------------------------------------------------- Step 1

def _step1_cost(c, prm, basis, yd, vd):
    """sum_t c_s + c_l + c_v of Sec. III-C, evaluated pointwise in t (P3 reading)."""
    W, Wd, Wdd = basis
    n = W.shape[1]
    cx, cy = c[:n], c[n:]
    x, y = W @ cx, W @ cy
    xd, yd_ = Wd @ cx, Wd @ cy
    xdd, ydd = Wdd @ cx, Wdd @ cy
    cs = xdd ** 2 + ydd ** 2
    cl = (ydd + prm.kp_lat * (y - yd) + prm.kv_lat * yd_) ** 2
    cv = (xdd + prm.kp_lon * (xd - vd)) ** 2
    return float(np.sum(cs + cl + cv))


def test_step1_closed_form_steady_state():
    """At-rest lateral motion with y_d = y0 stays at y0; cruise at v_d stays linear."""
    prm = _prm()
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    sc = _scene(0)
    sc.ego[:] = [0.0, 5.25, 17.0, 0.0, 0.0, 0.0]
    p = np.array([[5.25, 17.0]])
    xi = lower.step1(p, sc, prm, basis)[0]
    n = prm.n_coef
    t = np.arange(prm.m) * prm.dt
    np.testing.assert_allclose(basis[0] @ xi[n:], 5.25, atol=1e-9)
    np.testing.assert_allclose(basis[0] @ xi[:n], 17.0 * t, atol=1e-8)


@pytest.mark.parametrize("n_seg", [1, 2, 4])
def test_step1_is_constrained_minimiser(n_seg):
    """xi_bar satisfies A xi = b0 and no feasible direction lowers the cost."""
    prm = _prm(n_seg=n_seg, m=50)
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    sc = _scene(2)
    sc.ego[3:] = [0.4, -0.3, 0.2]
    p = sg.make_samples(9, sc, 5, n_seg)
    xb = lower.step1(p, sc, prm, basis)
    W, Wd, Wdd = basis
    n = prm.n_coef
    A1 = np.stack([W[0], Wd[0], Wdd[0]])
    Z = null_space(np.block([[A1, np.zeros_like(A1)], [np.zeros_like(A1), A1]]))
    rng = np.random.default_rng(0)
    for j in range(p.shape[0]):
        yd, vd = lower.setpoint_vectors(p[j:j + 1], prm.m, n_seg)
        np.testing.assert_allclose(A1 @ xb[j, :n], sc.ego[[0, 2, 4]], atol=1e-9)
        np.testing.assert_allclose(A1 @ xb[j, n:], sc.ego[[1, 3, 5]], atol=1e-9)
        f0 = _step1_cost(xb[j], prm, basis, yd[0], vd[0])
        # directional derivatives along the feasible subspace vanish
        eps = 1e-4
        for col in range(Z.shape[1]):
            dz = Z[:, col]
            fp = _step1_cost(xb[j] + eps * dz, prm, basis, yd[0], vd[0])
            fm = _step1_cost(xb[j] - eps * dz, prm, basis, yd[0], vd[0])
            assert abs(fp - fm) / (2 * eps) < 1e-5 * max(1.0, f0)
        for _ in range(5):
            dz = Z @ rng.normal(size=Z.shape[1])
            assert _step1_cost(xb[j] + 1e-2 * dz, prm, basis, yd[0], vd[0]) >= f0


def test_step1_null_space_method_agrees():
    """A second, independent solution method (null-space parametrisation)."""
    prm = _prm()
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    sc = _scene(1)
    p = sg.make_samples(3, sc, 4, 1)
    xb = lower.step1(p, sc, prm, basis)
    W, Wd, Wdd = basis
    n = prm.n_coef
    A1 = np.stack([W[0], Wd[0], Wdd[0]])
    for j in range(4):
        yd, vd = lower.setpoint_vectors(p[j:j + 1], prm.m, 1)
        for axis, bvec in ((0, sc.ego[[0, 2, 4]]), (1, sc.ego[[1, 3, 5]])):
            # least squares on stacked residual rows, restricted to A c = b
            if axis == 0:
                R = np.vstack([Wdd, Wdd + prm.kp_lon * Wd])
                tgt = np.concatenate([np.zeros(prm.m), prm.kp_lon * vd[0]])
            else:
                R = np.vstack([Wdd, Wdd + prm.kv_lat * Wd + prm.kp_lat * W])
                tgt = np.concatenate([np.zeros(prm.m), prm.kp_lat * yd[0]])
            c0 = np.linalg.lstsq(A1, bvec, rcond=None)[0]
            Z = null_space(A1)
            eta = np.linalg.lstsq(R @ Z, tgt - R @ c0, rcond=None)[0]
            c = c0 + Z @ eta
            np.testing.assert_allclose(xb[j, axis * n:(axis + 1) * n], c, rtol=1e-8, atol=1e-8)


def test_setpoint_segments():
    p = np.array([[1.0, 2.0, 3.0, 10.0, 20.0, 30.0]])
    yd, vd = lower.setpoint_vectors(p, 10, 3)
    assert list(yd[0]) == [1, 1, 1, 1, 2, 2, 2, 3, 3, 3]
    assert list(vd[0]) == [10, 10, 10, 10, 20, 20, 20, 30, 30, 30]


# --------------------------------------------------------------------------- Alg. 2 pieces

def _random_xi(prm, basis, sc, B=6, seed=1):
    p = sg.make_samples(seed, sc, B, prm.n_seg)
    return lower.step1(p, sc, prm, basis)


def test_obstacle_projection_lands_on_constraint_set():
    prm = _prm()
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    sc = _scene(4, seed=12, n_lanes=2)
    # slow vehicles ahead in both lanes, so some samples run into them
    sc.obstacles[:2] = [[20.0, 1.75, 4.0, 0.0, 2.8, 1.5], [30.0, 5.25, 2.0, 0.0, 2.8, 1.5]]
    xi = _random_xi(prm, basis, sc, B=8)
    da = np.full((8, prm.m), 1.0)
    h, _, parts = lower.alpha_d_step(xi, sc, prm, basis, da)
    x, y = lower.kinematics(xi, basis)[:2]
    xo, yo, a, b = lower.obstacle_trajectories(sc, prm.m, prm.dt)
    dx, dy = x[:, None] - xo[None], y[:, None] - yo[None]
    dist = np.sqrt((dx / a) ** 2 + (dy / b) ** 2)
    hx, hy = parts["hox"], parts["hoy"]
    hd = np.sqrt(((hx - xo[None]) / a) ** 2 + ((hy - yo[None]) / b) ** 2)
    np.testing.assert_allclose(hd, np.maximum(1.0, dist), rtol=1e-12)
    outside = dist >= 1.0
    assert outside.any() and (~outside).any()
    np.testing.assert_allclose(hx[outside], np.broadcast_to(x[:, None], dx.shape)[outside], atol=1e-9)
    np.testing.assert_allclose(hy[outside], np.broadcast_to(y[:, None], dy.shape)[outside], atol=1e-9)
    # clipped points lie on the ellipse along the same scaled ray from its centre
    cross = ((hx - xo[None]) / a) * (dy / b) - ((hy - yo[None]) / b) * (dx / a)
    dot = ((hx - xo[None]) / a) * (dx / a) + ((hy - yo[None]) / b) * (dy / b)
    assert np.abs(cross[~outside]).max() < 1e-9
    assert (dot[~outside] >= 0).all()


def test_velocity_acceleration_projection_invariants():
    """h_v, h_a are parallel to the trajectory's velocity / acceleration, within
    the speed and acceleration bounds, and satisfy the curvature bound of Table I."""
    prm = _prm(v_max=18.0, a_max=2.0, kappa_max=0.05)
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    sc = _scene(0, n_lanes=4)
    sc.ego[3:] = [1.5, 0.0, 0.0]
    xi = _random_xi(prm, basis, sc, B=16, seed=4)
    _, _, _, _, xdd, ydd = lower.kinematics(xi, basis)
    da_prev = np.minimum(np.hypot(xdd, ydd), prm.a_max)
    h, da, parts = lower.alpha_d_step(xi, sc, prm, basis, da_prev)
    x, y, xd, yd, xdd, ydd = lower.kinematics(xi, basis)
    hvx, hvy = parts["hv"]
    hax, hay = parts["ha"]
    sp = np.hypot(hvx, hvy)
    am = np.hypot(hax, hay)
    ok = parts["vmin_bar"] <= parts["vmax_bar"]
    assert ok.all()
    assert (sp >= prm.v_min - 1e-12).all() and (sp <= prm.v_max + 1e-12).all()
    assert (am <= prm.a_max + 1e-12).all()
    curv = np.abs(hax * hvy - hay * hvx) / sp ** 3
    assert (curv <= prm.kappa_max * (1 + 1e-9)).all()
    # the previous acceleration fits the curvature bound at the new speed
    # (Eq. d_reform_2 solved for d_v) unless capped by the speed bound
    S = np.abs(np.sin(parts["al_a"] - parts["al_v"]))
    uncapped = sp < prm.v_max - 1e-9
    assert (da_prev[uncapped] * S[uncapped] <= sp[uncapped] ** 2 * prm.kappa_max * (1 + 1e-9)).all()
    # directions preserved
    assert (np.abs(hvx * yd - hvy * xd) <= 1e-9 * sp * np.hypot(xd, yd) + 1e-12).all()
    assert (hvx * xd + hvy * yd >= 0).all()
    amag = np.hypot(xdd, ydd)
    nz = amag > 1e-9
    assert (np.abs(hax * ydd - hay * xdd)[nz] <= 1e-9 * (am * amag)[nz] + 1e-12).all()
    # the clip is inactive where the trajectory already satisfies all bounds
    speed = np.hypot(xd, yd)
    inside = (speed <= prm.v_max) & (speed >= parts["vmin_bar"]) & (amag <= parts["amax_bar"])
    np.testing.assert_allclose(hvx[inside], xd[inside], atol=1e-10)
    np.testing.assert_allclose(hax[inside], xdd[inside], atol=1e-10)


def test_vmin_bar_binds_at_low_speed():
    """Eq. (d_reform_2) solved for d_v: with the previous acceleration d_a and
    the angle between acceleration and velocity, a slow trajectory is sped up
    to exactly sqrt(d_a |sin(alpha_a - alpha_v)| / kappa_max)."""
    prm = _prm(kappa_max=0.2, v_min=0.1)
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    sc = _scene(0, n_lanes=4)
    sc.ego[:] = [0.0, 5.25, 2.0, 0.0, 0.0, 1.5]          # slow, accelerating sideways
    p = np.array([[8.75, 2.0]])
    xi = lower.step1(p, sc, prm, basis)
    _, _, xd, yd, xdd, ydd = lower.kinematics(xi, basis)
    da_prev = np.full_like(xd, 4.0)
    _, _, parts = lower.alpha_d_step(xi, sc, prm, basis, da_prev)
    S = np.abs(np.sin(np.arctan2(ydd, xdd) - np.arctan2(yd, xd)))
    bound = np.sqrt(da_prev * S / prm.kappa_max)
    active = (bound > np.hypot(xd, yd) + 1e-6) & (bound < prm.v_max) & (bound > prm.v_min)
    assert active.any()
    np.testing.assert_allclose(parts["d_v"][active], bound[active], rtol=1e-12)


def test_slack_nonnegative_and_exact_when_feasible():
    prm = _prm()
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    sc = _scene(0, n_lanes=2)
    xi = _random_xi(prm, basis, sc, B=10)
    F, G, A = lower.projection_operators(basis, 0)
    e = lower.lane_vector(sc, prm, prm.m)
    s = lower.slack_step(xi, G, e)
    assert (s >= 0).all()
    gx = xi @ G.T
    feas = gx <= e[None]
    np.testing.assert_allclose((gx - e[None] + s)[feas], 0.0, atol=1e-12)
    np.testing.assert_allclose(s[~feas], 0.0)


def _aug_lagrangian(xi, xi_bar, lam, h, s, F, G, e, rho):
    """Eq. (aug_lag) evaluated block by block."""
    return (0.5 * np.sum((xi - xi_bar) ** 2) - lam @ xi
            + 0.5 * rho * np.sum((F @ xi - h) ** 2)
            + 0.5 * rho * np.sum((G @ xi - e + s) ** 2))


def test_xi_step_minimises_augmented_lagrangian():
    prm = _prm(rho=0.7)
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    sc = _scene(3, seed=8)
    xb = _random_xi(prm, basis, sc, B=3)
    ops = lower.projection_operators(basis, sc.n_obs)
    F, G, A = ops
    e = lower.lane_vector(sc, prm, prm.m)
    rng = np.random.default_rng(2)
    lam = rng.normal(size=xb.shape)
    h = (xb @ F.T) + rng.normal(size=(3, F.shape[0]))
    s = np.abs(rng.normal(size=(3, G.shape[0])))
    b_eq = list(sc.ego[[0, 2, 4, 1, 3, 5]])
    xi = lower.xi_step(xb, lam, h, s, ops, e, b_eq, prm.rho)
    Z = null_space(A)
    for j in range(3):
        np.testing.assert_allclose(A @ xi[j], b_eq, atol=1e-9)
        f0 = _aug_lagrangian(xi[j], xb[j], lam[j], h[j], s[j], F, G, e, prm.rho)
        for col in range(Z.shape[1]):
            d = Z[:, col]
            fp = _aug_lagrangian(xi[j] + 1e-5 * d, xb[j], lam[j], h[j], s[j], F, G, e, prm.rho)
            fm = _aug_lagrangian(xi[j] - 1e-5 * d, xb[j], lam[j], h[j], s[j], F, G, e, prm.rho)
            assert abs(fp - fm) / 2e-5 < 1e-6 * max(1.0, abs(f0))


def test_fixed_point_when_feasible():
    """A feasible xi_bar with lambda^0 = 0 is returned unchanged by Alg. 2."""
    prm = _prm(v_max=60.0, a_max=50.0, kappa_max=50.0)
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    sc = _scene(2, n_lanes=3, obs_x=(400.0, 500.0))
    sc.ego[1] = sc.lane_centres()[1]
    p = np.array([[sc.lane_centres()[1], sc.ego[2]], [sc.lane_centres()[1], sc.ego[2] + 2.0]])
    xb = lower.step1(p, sc, prm, basis)
    r, _ = lower.score(xb, sc, prm, basis)
    assert (r == 0).all()
    xs = lower.project(xb, sc, prm, basis, iters=20)
    np.testing.assert_allclose(xs, xb, atol=1e-9)


def test_equality_rows_hold_every_iteration():
    prm = _prm()
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    sc = _scene(4, seed=21, n_lanes=2)
    xb = _random_xi(prm, basis, sc, B=5)
    _, _, A = lower.projection_operators(basis, sc.n_obs)
    b_eq = sc.ego[[0, 2, 4, 1, 3, 5]]
    for k in (1, 2, 7):
        xs = lower.project(xb, sc, prm, basis, iters=k)
        np.testing.assert_allclose(xs @ A.T, np.broadcast_to(b_eq, (5, 6)), atol=1e-9)


def test_convex_lane_case_limit():
    """No obstacles and loose kinematic bounds leave only the affine lane rows.
    Alg. 2 then drives the lane residual to zero (the role the paper gives the
    multipliers), and its displacement from xi_bar is a nonnegative combination
    of the violated constraints' normals plus the equality rows (stationarity of
    Eq. split_xy with lambda accumulated by Eq. update_lagrange).  Because the
    slack step never lets a multiplier shrink, the limit is feasible but need
    not be the exact Euclidean projection: its distance is bounded below by the
    projection computed independently with SLSQP."""
    from scipy.optimize import nnls
    prm = _prm(m=40, v_max=80.0, a_max=80.0, kappa_max=1e3, v_min=0.0)
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    sc = _scene(0, n_lanes=2)
    sc.ego[1] = 5.0
    p = np.array([[8.5, 15.0]])     # lateral target beyond the road edge
    xb = lower.step1(p, sc, prm, basis)
    _, G, A = lower.projection_operators(basis, 0)
    e = lower.lane_vector(sc, prm, prm.m)
    b_eq = sc.ego[[0, 2, 4, 1, 3, 5]]
    assert (xb @ G.T > e[None] + 1e-3).any()
    res = minimize(lambda z: 0.5 * np.sum((z - xb[0]) ** 2), xb[0], jac=lambda z: z - xb[0],
                   method="SLSQP",
                   constraints=[dict(type="eq", fun=lambda z: A @ z - b_eq, jac=lambda z: A),
                                dict(type="ineq", fun=lambda z: e - G @ z, jac=lambda z: -G)],
                   options=dict(ftol=1e-14, maxiter=500))
    assert res.success
    xs = lower.project(xb, sc, prm, basis, iters=2000)[0]
    assert (G @ xs - e).max() <= 1e-6                       # feasible
    np.testing.assert_allclose(A @ xs, b_eq, atol=1e-9)
    assert 0.5 * np.sum((xs - xb[0]) ** 2) >= res.fun - 1e-9  # projection is closest
    cone = np.hstack([-G.T, -A.T, A.T])
    _, resid = nnls(cone, xs - xb[0])
    assert resid <= 1e-7 * max(1.0, np.abs(xs - xb[0]).max())


def test_projection_reduces_residual_on_static_obstacles():
    """Sec. V-B, Fig. 5: the projection lowers the constraint residual."""
    prm = _prm(m=80, inner_iters=60)
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    sc = _scene(5, seed=33, n_lanes=3, obs_vx=(0.0, 0.0), obs_x=(15.0, 60.0))
    xb = _random_xi(prm, basis, sc, B=40, seed=6)
    r0, _ = lower.score(xb, sc, prm, basis)
    xs = lower.project(xb, sc, prm, basis)
    r1, _ = lower.score(xs, sc, prm, basis)
    assert r1.mean() < 0.5 * r0.mean()


def test_batch_structure():
    """B=1 equals the batch row; permuting samples permutes results."""
    prm = _prm(inner_iters=8)
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    sc = _scene(3, seed=2)
    p = sg.make_samples(4, sc, 6, 1)
    xs, r, cu = lower.solve(p, sc, prm, basis)
    xs1, r1, _ = lower.solve(p[3:4], sc, prm, basis)
    np.testing.assert_allclose(xs1[0], xs[3], rtol=1e-12, atol=1e-11)
    perm = np.array([5, 2, 0, 4, 1, 3])
    xsp, rp, cup = lower.solve(p[perm], sc, prm, basis)
    np.testing.assert_allclose(xsp, xs[perm], rtol=1e-12, atol=1e-11)


# --------------------------------------------------------------------------- scoring

def test_score_constant_speed_closed_form():
    """Straight cruise at v along a lane centre: only the speed row can fire."""
    prm = _prm(v_max=20.0)
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    sc = _scene(0, n_lanes=2)
    n = prm.n_coef
    tf = (prm.m - 1) * prm.dt
    k = np.arange(n) / (n - 1)
    for v in (15.0, 23.0):
        xi = np.concatenate([v * tf * k, np.full(n, 1.75)])[None]
        r, cu = lower.score(xi, sc, prm, basis)
        np.testing.assert_allclose(r[0], prm.m * max(0.0, v - 20.0), rtol=1e-10)
        np.testing.assert_allclose(cu[0], prm.m * (v - 20.0) ** 2, rtol=1e-10)


def test_score_lane_and_collision_rows():
    prm = _prm(v_max=30.0)
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    n = prm.n_coef
    tf = (prm.m - 1) * prm.dt
    k = np.arange(n) / (n - 1)
    sc = _scene(0, n_lanes=2)
    # 0.5 m beyond the upper lane bound at every step
    ub = 2 * 3.5 - prm.lane_margin
    xi = np.concatenate([10.0 * tf * k, np.full(n, ub + 0.5)])[None]
    r, _ = lower.score(xi, sc, prm, basis)
    np.testing.assert_allclose(r[0], prm.m * 0.5, rtol=1e-10)
    # an obstacle moving with the ego, centred 1 m ahead on the same line:
    # 1 - (1/a)^2 at every step
    sc.obstacles = np.array([[1.0, 1.75, 10.0, 0.0, 2.8, 1.5]])
    xi = np.concatenate([10.0 * tf * k, np.full(n, 1.75)])[None]
    r, _ = lower.score(xi, sc, prm, basis)
    np.testing.assert_allclose(r[0], prm.m * (1 - 1 / 2.8 ** 2), rtol=1e-10)


def test_score_curvature_row_on_constant_lateral_acceleration():
    """x = v t, y = y0 + g t^2 / 2: curvature g v / (v^2 + g^2 t^2)^1.5."""
    prm = _prm(v_max=40.0, a_max=10.0, kappa_max=0.02)
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    n = prm.n_coef
    tf = (prm.m - 1) * prm.dt
    k = np.arange(n, dtype=float)
    d = n - 1
    v, g = 8.0, 2.0
    cx = v * tf * k / d
    cy = 3.0 + 0.5 * g * tf ** 2 * k * (k - 1) / (d * (d - 1))
    sc = _scene(0, n_lanes=8)
    r, _ = lower.score(np.concatenate([cx, cy])[None], sc, prm, basis)
    t = np.arange(prm.m) * prm.dt
    kap = g * v / (v ** 2 + (g * t) ** 2) ** 1.5
    np.testing.assert_allclose(r[0], np.maximum(0, kap - 0.02).sum(), rtol=1e-9)
