"""Pins of the oracle with goal entries in p: Eq. behaviour_param's x_f, y_f,
which enter the affine equality rows of Eq. final_boundary,
(x(t_f), y(t_f), ydot(t_f)) = (x_f, y_f, 0), through b(p) (Sec. IV-A: the
set-points enter the cost, the goal positions the equality constraints).

Checked against: an exact closed form (a goal consistent with steady cruise
is met by the straight constant-speed line), feasibility and stationarity of
the Step-1 cost along null(A) written term by term, a second Step-1 solver
(null-space least squares), the terminal rows at every Alg. 2 iteration,
the row-by-row restatement of Alg. 2, central differences of the layer, and
the support and moments of the first-iteration draw."""
import numpy as np
import pytest
from scipy.linalg import null_space

import test_oracle_alg2_rowwise as ta
from oracle import lower, upper
from oracle.basis import bernstein
from paper_2212_02224_gb300 import scenegen as sg


def _prm(**kw):
    p = sg.Params(m=60, n_coef=11, inner_iters=30, goal=True)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _tf(prm):
    return (prm.m - 1) * prm.dt


def _goal_samples(seed, sc, prm, B):
    return sg.make_samples(seed, sc, B, prm.n_seg, goal_tf=_tf(prm))


def test_goal_layout_and_sizes():
    prm = _prm(n_seg=4)
    assert prm.d_p == 10
    sc = sg.make_scene(3, n_lanes=3, n_obs=0)
    p = _goal_samples(1, sc, prm, 50)
    assert p.shape == (50, 10)
    assert set(np.unique(p[:, 9])) <= set(sc.lane_centres())
    lo, hi = sc.ego[0] + 5.0 * _tf(prm), sc.ego[0] + 25.0 * _tf(prm)
    assert (p[:, 8] >= lo).all() and (p[:, 8] <= hi).all()


def test_goal_cruise_closed_form():
    """Ego on a lane centre at 17 m/s, set-points y_d = y0, v_d = 17 and the
    goal (x0 + 17 t_f, y0): the straight line at constant speed costs nothing
    and meets every row, so Step 1 returns it exactly."""
    prm = _prm()
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    sc = sg.make_scene(2, n_lanes=3, n_obs=0)
    sc.ego[:] = [3.0, 5.25, 17.0, 0.0, 0.0, 0.0]
    p = np.array([[5.25, 17.0, 3.0 + 17.0 * _tf(prm), 5.25]])
    xi = lower.step1(p, sc, prm, basis)[0]
    n = prm.n_coef
    t = np.arange(prm.m) * prm.dt
    np.testing.assert_allclose(basis[0] @ xi[:n], 3.0 + 17.0 * t, atol=1e-8)
    np.testing.assert_allclose(basis[0] @ xi[n:], 5.25, atol=1e-9)


@pytest.mark.parametrize("n_seg", [1, 4])
def test_goal_step1_feasible_and_stationary(n_seg):
    """xi_bar meets all eight equality rows and no feasible direction lowers
    the Step-1 cost written term by term (c_s + c_l + c_v per t)."""
    prm = _prm(n_seg=n_seg, m=50)
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    W, Wd, Wdd = basis
    sc = sg.make_scene(4, n_lanes=3, n_obs=0)
    sc.ego[3:] = [0.4, -0.3, 0.2]
    p = _goal_samples(9, sc, prm, 5)
    xb = lower.step1(p, sc, prm, basis)
    n = prm.n_coef
    Ax = np.stack([W[0], Wd[0], Wdd[0], W[-1]])
    Ay = np.stack([W[0], Wd[0], Wdd[0], W[-1], Wd[-1]])
    Z = null_space(np.block([[Ax, np.zeros((4, n))], [np.zeros((5, n)), Ay]]))
    assert Z.shape[1] == 2 * n - 9
    for j in range(p.shape[0]):
        np.testing.assert_allclose(Ax @ xb[j, :n], [*sc.ego[[0, 2, 4]], p[j, 2 * n_seg]], atol=1e-8)
        np.testing.assert_allclose(Ay @ xb[j, n:], [*sc.ego[[1, 3, 5]], p[j, 2 * n_seg + 1], 0.0],
                                   atol=1e-8)
        yd, vd = lower.setpoint_vectors(p[j:j + 1], prm.m, n_seg)

        def cost(c):
            x, y = W @ c[:n], W @ c[n:]
            xd, yd_ = Wd @ c[:n], Wd @ c[n:]
            xdd, ydd = Wdd @ c[:n], Wdd @ c[n:]
            return float(np.sum(xdd ** 2 + ydd ** 2
                                + (ydd + prm.kp_lat * (y - yd[0]) + prm.kv_lat * yd_) ** 2
                                + (xdd + prm.kp_lon * (xd - vd[0])) ** 2))
        f0 = cost(xb[j])
        eps = 1e-4
        for col in range(Z.shape[1]):
            dz = Z[:, col]
            assert abs(cost(xb[j] + eps * dz) - cost(xb[j] - eps * dz)) / (2 * eps) < 1e-5 * max(1.0, f0)


def test_goal_step1_null_space_method_agrees():
    """A second solver: least squares of the stacked cost rows over
    {c : A c = b(p)} by a particular solution plus null(A)."""
    prm = _prm()
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    W, Wd, Wdd = basis
    n = prm.n_coef
    sc = sg.make_scene(1, n_lanes=4, n_obs=0)
    p = _goal_samples(3, sc, prm, 4)
    xb = lower.step1(p, sc, prm, basis)
    for j in range(4):
        yd, vd = lower.setpoint_vectors(p[j:j + 1], prm.m, 1)
        for axis in (0, 1):
            if axis == 0:
                A = np.stack([W[0], Wd[0], Wdd[0], W[-1]])
                b = [*sc.ego[[0, 2, 4]], p[j, 2]]
                R = np.vstack([Wdd, Wdd + prm.kp_lon * Wd])
                tgt = np.concatenate([np.zeros(prm.m), prm.kp_lon * vd[0]])
            else:
                A = np.stack([W[0], Wd[0], Wdd[0], W[-1], Wd[-1]])
                b = [*sc.ego[[1, 3, 5]], p[j, 3], 0.0]
                R = np.vstack([Wdd, Wdd + prm.kv_lat * Wd + prm.kp_lat * W])
                tgt = np.concatenate([np.zeros(prm.m), prm.kp_lat * yd[0]])
            c0 = np.linalg.lstsq(A, b, rcond=None)[0]
            Z = null_space(A)
            eta = np.linalg.lstsq(R @ Z, tgt - R @ c0, rcond=None)[0]
            np.testing.assert_allclose(xb[j, axis * n:(axis + 1) * n], c0 + Z @ eta, rtol=1e-8,
                                       atol=1e-7)


def test_goal_rows_hold_every_iteration():
    """x(t_f) = x_f, y(t_f) = y_f and ydot(t_f) = 0 for every iterate of Alg. 2
    (the xi-step of Eq. split_xy keeps A xi = b(p) with each sample's goal)."""
    prm = _prm()
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    W, Wd, _ = basis
    n = prm.n_coef
    sc = sg.make_scene(21, n_lanes=2, n_obs=4)
    p = _goal_samples(5, sc, prm, 6)
    xb = lower.step1(p, sc, prm, basis)
    for k in (1, 2, 9):
        xs = lower.project(xb, sc, prm, basis, iters=k, p=p)
        np.testing.assert_allclose(xs[:, :n] @ W[-1], p[:, 2], atol=1e-8)
        np.testing.assert_allclose(xs[:, n:] @ W[-1], p[:, 3], atol=1e-9)
        np.testing.assert_allclose(xs[:, n:] @ Wd[-1], 0.0, atol=1e-9)
        np.testing.assert_allclose(xs[:, :n] @ W[0], sc.ego[0], atol=1e-9)


def test_goal_project_needs_p():
    prm = _prm()
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    sc = sg.make_scene(21, n_lanes=2, n_obs=1)
    xb = lower.step1(_goal_samples(5, sc, prm, 2), sc, prm, basis)
    with pytest.raises(ValueError):
        lower.project(xb, sc, prm, basis, iters=1)


@pytest.mark.parametrize("iters", [1, 2])
def test_goal_project_matches_rowwise_restatement(iters):
    """The row-by-row statement of Alg. 2 with the terminal rows in its own
    equality system agrees with lower.project."""
    prm, sc, p = ta._setup()
    prm.goal = True
    tf = (prm.m - 1) * prm.dt
    p = np.array([[p[0, 0], p[0, 1], 14.0 * tf, 5.25]])
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    xb = lower.step1(p, sc, prm, basis)
    got = lower.project(xb, sc, prm, basis, iters=iters, p=p)[0]
    want = ta._Sample(xb[0], sc, prm, goal=(p[0, 2], p[0, 3])).run(iters)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-9 * max(1.0, np.abs(want).max()))


def test_goal_layer_vjp_matches_central_differences():
    prm = sg.Params(m=60, n_coef=11, n_seg=2, goal=True)
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    s = sg.Stream(7)
    B = 3
    p = np.concatenate([s.uniform(0.0, 14.0, B * 2).reshape(B, 2), s.uniform(5.0, 25.0, B * 2).reshape(B, 2),
                        s.uniform(20.0, 70.0, B)[:, None], s.uniform(0.0, 14.0, B)[:, None]], axis=1)
    b0 = np.stack([s.uniform(-5, 5, B), s.uniform(0, 14, B), s.uniform(5, 20, B),
                   s.uniform(-1, 1, B), s.uniform(-2, 2, B), s.uniform(-1, 1, B)], axis=1)
    g = s.normal(0.0, 1.0, B * 2 * prm.n_coef).reshape(B, 2 * prm.n_coef)
    gp, gb = lower.step1_layer_vjp(g, prm, basis)
    loss = lambda pp, bb: float(np.sum(g * lower.step1_layer(pp, bb, prm, basis)))
    h = 1e-3
    fd_p = np.zeros_like(p)
    for j in range(B):
        for a in range(p.shape[1]):
            e = np.zeros_like(p)
            e[j, a] = h
            fd_p[j, a] = (loss(p + e, b0) - loss(p - e, b0)) / (2 * h)
    fd_b = np.zeros_like(b0)
    for j in range(B):
        for a in range(6):
            e = np.zeros_like(b0)
            e[j, a] = h
            fd_b[j, a] = (loss(p, b0 + e) - loss(p, b0 - e)) / (2 * h)
    np.testing.assert_allclose(gp, fd_p, rtol=1e-6, atol=1e-6 * np.abs(fd_p).max())
    np.testing.assert_allclose(gb, fd_b, rtol=1e-6, atol=1e-6 * np.abs(fd_b).max())


def test_goal_layer_with_shared_state_is_step1():
    prm = _prm(n_seg=2)
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    sc = sg.make_scene(6, n_lanes=3, n_obs=0)
    p = _goal_samples(4, sc, prm, 5)
    b0 = np.repeat(np.asarray(sc.ego, float)[None], 5, axis=0)
    np.testing.assert_allclose(lower.step1_layer(p, b0, prm, basis), lower.step1(p, sc, prm, basis),
                               rtol=1e-12, atol=1e-9)


def test_goal_initial_draws_and_moments():
    """First-iteration draw with goal entries: x_f = x0 + U[v_des_lo, v_des_hi] t_f
    and y_f on lane centres, with the moments initial_moments states."""
    prm = sg.Params(n_seg=2, goal=True, m=100)
    sc = sg.make_scene(1, n_lanes=4, n_obs=0)
    sc.ego[0] = 2.0
    p = upper.draw_initial(100000, sc, prm, 3, 0)
    tf = _tf(prm)
    assert p.shape == (100000, 6)
    assert set(np.unique(p[:, 5])) == set(sc.lane_centres())
    assert p[:, 4].min() >= 2.0 + prm.v_des_lo * tf and p[:, 4].max() <= 2.0 + prm.v_des_hi * tf
    mu, sigma = upper.initial_moments(sc, prm)
    N = p.shape[0]
    sd = np.sqrt(np.diag(sigma))
    # six standard errors of the sample mean and of the sample covariance
    assert (np.abs(p.mean(0) - mu) <= 6 * sd / np.sqrt(N)).all()
    assert (np.abs(np.cov(p.T) - sigma) <= 6 * np.sqrt(2.0) * np.outer(sd, sd) / np.sqrt(N)).all()
    # the goal entries use words 4 and 5 of the draw, independent of the set-points
    assert abs(np.corrcoef(p[:, 4], p[:, 2])[0, 1]) < 0.01


def test_goal_plan_runs_and_meets_goal_rows():
    """Alg. 1 with goal entries: the returned best pair meets its own goal."""
    prm = sg.Params(m=40, n_coef=11, n_seg=1, goal=True, inner_iters=10, outer_iters=2,
                    n_elite_c=12, n_elite=4)
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    sc = sg.make_scene(8, n_lanes=3, n_obs=3)
    out = upper.plan(sc, prm, 32, seed=5, basis=basis)
    n = prm.n_coef
    assert len(out["p"]) == 4
    np.testing.assert_allclose(basis[0][-1] @ out["xi"][:n], out["p"][2], atol=1e-8)
    np.testing.assert_allclose(basis[0][-1] @ out["xi"][n:], out["p"][3], atol=1e-9)
