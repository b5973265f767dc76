"""Lower-level trajectory optimisation, FP64, batched over samples p_j.

Follows Sec. III-C (cost and constraints), Alg. 1 Step 1 with Eq. (over_2),
Appendix A (Table I, Eqs. sphere_proposed .. lane_reform, the augmented
Lagrangian aug_lag) and Alg. 2 (Eqs. split_xy .. update_lagrange).  All
matrices are assembled literally (F stacks W once per obstacle, G = [W; -W]
on the y block) so the code can be read against the paper.

Shapes: B samples, m timesteps, n coefficients per axis, N obstacles.
xi is (B, 2n) = [c_x | c_y].

Readings of the paper adopted here:
  * PD tracking (Eq. cost, printed with unbalanced parentheses): stable
    tracking c_l = (ydd + kp (y - y_d) + kv yd)^2, c_v = (xdd + kp (xd - v_d))^2,
    weights of c_s, c_l, c_v all one.
  * Equality constraints: the initial state b0 (Eq. boundary_cond_initial)
    and, when p carries goal entries (prm.goal, Eq. behaviour_param's x_f,
    y_f), the final rows of Eq. final_boundary: x(t_f) = x_f on the x axis,
    y(t_f) = y_f and ydot(t_f) = 0 on the y axis.  The goal positions enter
    only b(p) (Sec. IV-A, after Eq. lower_eq); the paper's MPC-Bi-Level runs
    use set-points alone (goal off).
  * Ellipse: a, b are the semi-axes used in Table I's collision expression;
    h_y uses y_o + b d sin(alpha) (the printed "x_o + a d sin" is a slip).
  * v_min-bar of Eq. (clip_d_v): max(v_min, sqrt(d_a |sin(a_a - a_v)| / kappa_max)),
    i.e. Eq. (d_reform_2) solved for d_v; v_max-bar from Eq. (d_reform_3),
    equal to v_max on a straight road.  clip(x, lo, hi) = min(max(x, lo), hi).
  * a_max-bar (Eq. clip_d_a) when |sin| = 0: a_max.
  * atan2(0, 0) = 0.
  * Slack (Eq. update_slack, printed sign garbled): s = max(0, e - G xi).
  * Multipliers (Eq. update_lagrange, operator missing between the terms):
    lambda <- lambda - rho/2 F^T (F xi - h) - rho/2 G^T (G xi - e + s).
  * Alg. 2 start: xi^0 = xi_bar, lambda^0 = 0, d_a^{-1} = min(|a(xi^0)|, a_max),
    then alpha^0, d^0, s^0 from xi^0 by the same steps as an iteration.

Pins: Step 1, the projections, the slack, the xi-step and the scoring are
pinned by closed forms and invariants (tests/test_oracle_lower.py).  The
iteration of Alg. 2 as a whole -- including the multiplier step rho/2 of
Eq. update_lagrange and the curvature lag kappa(^k xi) of Eq. clip_d_v, which
no invariant fixes -- is pinned by a second, row-by-row statement of the
algorithm written independently (per-row F/G assembly, math.atan2 projections,
a null-space xi-step) on a scene where every block is active
(tests/test_oracle_alg2_rowwise.py).  Both statements follow the same readings
of the garbled passages listed above; those readings are choices, not pins.
"""
from __future__ import annotations

import numpy as np


# ----------------------------------------------------------------------------
# behavioural inputs -> set-point vectors
# ----------------------------------------------------------------------------

def segment_lengths(m: int, n_seg: int):
    """Contiguous segments; with m = n_seg*q + r the first r get q+1 steps."""
    q, r = divmod(m, n_seg)
    return [q + 1 if j < r else q for j in range(n_seg)]


def setpoint_vectors(p: np.ndarray, m: int, n_seg: int):
    """y_d, v_d (B, m): each segment's set-point repeated over its steps
    (Sec. III-C, the sentence after the cost terms; p per Eq. behaviour_param,
    p = [y_d,1..n_seg, v_d,1..n_seg(, x_f, y_f)])."""
    seg_of_t = np.repeat(np.arange(n_seg), segment_lengths(m, n_seg))
    return p[:, :n_seg][:, seg_of_t], p[:, n_seg:2 * n_seg][:, seg_of_t]


def lane_bounds(scene, prm):
    """y_lb, y_ub of Table I's lane-boundary row (straight road, margin inside)."""
    return prm.lane_margin, scene.n_lanes * scene.lane_width - prm.lane_margin


def road_at(scene, prm, x):
    """Road curvature kappa(x) and lane limits y_lb(x), y_ub(x) at arc length x
    (any shape), Table I's centripetal and lane-boundary rows on a road given
    in the Frenet frame.  With a knot table (s, kappa, lb, ub): linear
    interpolation in x + road_origin, constant beyond the end knots, limits =
    edges moved inwards by the lane margin.  Without one: kappa_road and the straight
    lanes of lane_bounds."""
    x = np.asarray(x, dtype=np.float64) + float(getattr(scene, "road_origin", 0.0))
    road = np.asarray(getattr(scene, "road", np.zeros((0, 4))), dtype=np.float64).reshape(-1, 4)
    if road.shape[0] == 0:
        ylb, yub = lane_bounds(scene, prm)
        return (np.full(x.shape, float(scene.kappa_road)), np.full(x.shape, ylb),
                np.full(x.shape, yub))
    sk = road[:, 0]
    kappa = np.interp(x, sk, road[:, 1])
    ylb = np.interp(x, sk, road[:, 2]) + prm.lane_margin
    yub = np.interp(x, sk, road[:, 3]) - prm.lane_margin
    return kappa, ylb, yub


def obstacle_trajectories(scene, m: int, dt: float):
    """x_o,i(t), y_o,i(t), (N, m): constant-velocity neighbours."""
    t = np.arange(m) * dt
    ob = np.asarray(scene.obstacles, dtype=np.float64).reshape(-1, 6)
    xo = ob[:, 0:1] + ob[:, 2:3] * t[None, :]
    yo = ob[:, 1:2] + ob[:, 3:4] * t[None, :]
    return xo, yo, ob[:, 4:5], ob[:, 5:6]


# ----------------------------------------------------------------------------
# Step 1: QP without inequalities (Alg. 1 line 7, Eq. over_2)
# ----------------------------------------------------------------------------

def step1_cost_matrices(basis, prm):
    """Per-axis (Q, L): cost sum_t c_s + c_v (x) and c_s + c_l (y) as
    1/2 c^T Q c + q^T c with q = -2 k L^T (set-point)."""
    W, Wd, Wdd = basis
    Lx = Wdd + prm.kp_lon * Wd
    Ly = Wdd + prm.kv_lat * Wd + prm.kp_lat * W
    Qx = 2.0 * (Wdd.T @ Wdd + Lx.T @ Lx)
    Qy = 2.0 * (Wdd.T @ Wdd + Ly.T @ Ly)
    return (Qx, Lx), (Qy, Ly)


def initial_rows(basis):
    """A of one axis: position, velocity and acceleration at t0."""
    W, Wd, Wdd = basis
    return np.stack([W[0], Wd[0], Wdd[0]])


def equality_rows(basis, goal: bool = False):
    """(A_x, A_y) of Eq. lower_eq: the initial rows of Eq. boundary_cond_initial
    and, with goal entries in p, the final rows of Eq. final_boundary
    (x(t_f) on the x axis; y(t_f) and ydot(t_f) on the y axis)."""
    W, Wd, Wdd = basis
    A0 = initial_rows(basis)
    if not goal:
        return A0, A0
    return np.vstack([A0, W[-1]]), np.vstack([A0, W[-1], Wd[-1]])


def equality_rhs(p, scene, prm):
    """b(p) of Eq. lower_eq per axis, (B, ne_x) and (B, ne_y): b0 of the ego
    state, then x_f (x axis) and y_f, 0 (y axis) from the goal entries of p."""
    p = np.atleast_2d(np.asarray(p, dtype=np.float64))
    B = p.shape[0]
    x0, y0, vx0, vy0, ax0, ay0 = np.asarray(scene.ego, dtype=np.float64)
    bx = np.tile([x0, vx0, ax0], (B, 1))
    by = np.tile([y0, vy0, ay0], (B, 1))
    if getattr(prm, "goal", False):
        ns = prm.n_seg
        bx = np.column_stack([bx, p[:, 2 * ns]])
        by = np.column_stack([by, p[:, 2 * ns + 1], np.zeros(B)])
    return bx, by


def kkt_solve(Q, A, rhs_top, rhs_bot):
    """Solve [[Q, A^T], [A, 0]] [z; mu] = [rhs_top; rhs_bot] for B columns
    (LU with partial pivoting via numpy); rhs_bot is (ne,), shared by the
    columns, or (B, ne), one per column.  Returns z (B, n)."""
    n, ne = Q.shape[0], A.shape[0]
    B = rhs_top.shape[0]
    K = np.zeros((n + ne, n + ne))
    K[:n, :n] = Q
    K[:n, n:] = A.T
    K[n:, :n] = A
    bot = np.asarray(rhs_bot, dtype=np.float64)
    bot = np.broadcast_to(bot if bot.ndim == 2 else bot[None, :], (B, ne))
    R = np.concatenate([rhs_top.T, bot.T], axis=0)
    return np.linalg.solve(K, R)[:n].T


def step1(p, scene, prm, basis):
    """xi_bar (B, 2n): the equality-constrained QP of Alg. 1 line 7 for each p_j."""
    m = basis[0].shape[0]
    p = np.atleast_2d(p)
    yd, vd = setpoint_vectors(p, m, prm.n_seg)
    (Qx, Lx), (Qy, Ly) = step1_cost_matrices(basis, prm)
    Ax, Ay = equality_rows(basis, getattr(prm, "goal", False))
    bx, by = equality_rhs(p, scene, prm)
    qx = -2.0 * prm.kp_lon * (vd @ Lx)          # (B, n) rows are (L^T v_d)^T
    qy = -2.0 * prm.kp_lat * (yd @ Ly)
    cx = kkt_solve(Qx, Ax, -qx, bx)
    cy = kkt_solve(Qy, Ay, -qy, by)
    return np.concatenate([cx, cy], axis=1)


def step1_layer(p, b0, prm, basis):
    """The Step-1 QP as a layer of the learned sampler (Sec. IV, choice of the
    differentiable optimizer: the convex cost of Alg. 1 line 7 and the equality
    constraints, inequalities ignored), with a separate initial state per row:
    p (B, d_p), b0 (B, 6) = (x, y, vx, vy, ax, ay) -> xi (B, 2n)."""
    p = np.atleast_2d(np.asarray(p, dtype=np.float64))
    b0 = np.atleast_2d(np.asarray(b0, dtype=np.float64))
    m = basis[0].shape[0]
    goal = getattr(prm, "goal", False)
    ns = prm.n_seg
    yd, vd = setpoint_vectors(p, m, ns)
    (Qx, Lx), (Qy, Ly) = step1_cost_matrices(basis, prm)
    Ax, Ay = equality_rows(basis, goal)
    qx = -2.0 * prm.kp_lon * (vd @ Lx)
    qy = -2.0 * prm.kp_lat * (yd @ Ly)
    cx, cy = [], []
    for j in range(len(p)):
        bx, by = list(b0[j, [0, 2, 4]]), list(b0[j, [1, 3, 5]])
        if goal:
            bx += [p[j, 2 * ns]]
            by += [p[j, 2 * ns + 1], 0.0]
        cx.append(kkt_solve(Qx, Ax, -qx[j:j + 1], bx)[0])
        cy.append(kkt_solve(Qy, Ay, -qy[j:j + 1], by)[0])
    return np.concatenate([np.stack(cx), np.stack(cy)], axis=1)


def step1_layer_vjp(g, prm, basis):
    """Vector-Jacobian product of step1_layer: g = dL/dxi (B, 2n) ->
    (dL/dp (B, d_p), dL/db0 (B, 6)).  Implicit differentiation of the KKT
    system K [z; mu] = [-q; b] (K symmetric): [u; w] = K^-1 [g_z; 0] gives
    dL/d(-q) = u and dL/db = w; -q = 2 k L^T s(p) with s the set-point vector,
    so dL/ds = 2 k L u and each entry of p collects dL/ds over its segment.
    A goal entry of p (x_f, y_f) is an entry of b: its gradient is the matching
    entry of w."""
    g = np.atleast_2d(np.asarray(g, dtype=np.float64))
    n = basis[0].shape[1]
    m = basis[0].shape[0]
    goal = getattr(prm, "goal", False)
    (Qx, Lx), (Qy, Ly) = step1_cost_matrices(basis, prm)
    Ax, Ay = equality_rows(basis, goal)
    seg_of_t = np.repeat(np.arange(prm.n_seg), segment_lengths(m, prm.n_seg))
    B = len(g)
    grad_p = np.zeros((B, 2 * prm.n_seg + (2 if goal else 0)))
    grad_b = np.zeros((B, 6))
    for axis, (Q, L, k, off, A) in enumerate([(Qx, Lx, prm.kp_lon, prm.n_seg, Ax),
                                              (Qy, Ly, prm.kp_lat, 0, Ay)]):
        ne = A.shape[0]
        K = np.zeros((n + ne, n + ne))
        K[:n, :n] = Q
        K[:n, n:] = A.T
        K[n:, :n] = A
        rhs = np.concatenate([g[:, axis * n:(axis + 1) * n].T, np.zeros((ne, B))], axis=0)
        uw = np.linalg.solve(K, rhs)            # K is symmetric: K^-T = K^-1
        u, w = uw[:n].T, uw[n:].T               # (B, n), (B, 3)
        ds = 2.0 * k * (u @ L.T)                # (B, m)
        for j in range(prm.n_seg):
            grad_p[:, off + j] = ds[:, seg_of_t == j].sum(axis=1)
        grad_b[:, [axis, axis + 2, axis + 4]] = w[:, :3]
        if goal:
            grad_p[:, 2 * prm.n_seg + axis] = w[:, 3]     # x_f (x axis) or y_f (y axis)
    return grad_p, grad_b


# ----------------------------------------------------------------------------
# Alg. 2: batch projection
# ----------------------------------------------------------------------------

def projection_operators(basis, n_obs: int, goal: bool = False):
    """F (Eq. after lane_reform), G (lane rows, y block) and A_eq, literal."""
    W, Wd, Wdd = basis
    m, n = W.shape
    Fax = np.vstack([W] * n_obs + [Wd, Wdd])
    Z = np.zeros_like(Fax)
    F = np.block([[Fax, Z], [Z, Fax]])
    Zm = np.zeros_like(W)
    G = np.block([[Zm, W], [Zm, -W]])
    Ax, Ay = equality_rows(basis, goal)
    A = np.block([[Ax, np.zeros((Ax.shape[0], n))], [np.zeros((Ay.shape[0], n)), Ay]])
    return F, G, A


def _angle(sy, cx):
    """atan2 with the convention atan2(0, 0) = 0 whatever the zero signs."""
    return np.where((sy == 0) & (cx == 0), 0.0, np.arctan2(sy, cx))


def kinematics(xi, basis):
    """x, y, xd, yd, xdd, ydd, each (B, m), through Eq. (param)."""
    W, Wd, Wdd = basis
    n = W.shape[1]
    cx, cy = xi[:, :n], xi[:, n:]
    return cx @ W.T, cy @ W.T, cx @ Wd.T, cy @ Wd.T, cx @ Wdd.T, cy @ Wdd.T


def alpha_d_step(xi, scene, prm, basis, da_prev, x_prev=None):
    """Eq. (split_alpha_o) followed by the clips (clip_d_o), (clip_d_v), (clip_d_a).

    The unconstrained minimiser of ||F xi - h(alpha, d)||^2 makes every block
    residual zero: for obstacle i, (x - x_o, y - y_o) = (a d cos(al), b d sin(al))
    gives al = atan2((y - y_o)/b, (x - x_o)/a), d = its scaled length; for the
    velocity and acceleration blocks the polar angle and magnitude.
    The road curvature of v_max-bar is kappa(^k xi) as printed in Eq. (clip_d_v):
    taken at the positions x_prev of the previous iterate (default: of xi).
    Returns h (B, rows of F), the clipped d_a (B, m) and the pieces as a dict.
    """
    W = basis[0]
    m = W.shape[0]
    x, y, xd, yd, xdd, ydd = kinematics(xi, basis)
    xo, yo, a, b = obstacle_trajectories(scene, m, prm.dt)

    # obstacles, (B, N, m)
    dx = x[:, None, :] - xo[None]
    dy = y[:, None, :] - yo[None]
    al_o = _angle(dy / b[None], dx / a[None])
    d_o = np.sqrt((dx / a[None]) ** 2 + (dy / b[None]) ** 2)
    d_o = np.maximum(1.0, d_o)                                   # clip_d_o
    hox = xo[None] + a[None] * d_o * np.cos(al_o)
    hoy = yo[None] + b[None] * d_o * np.sin(al_o)

    # velocity and acceleration, (B, m)
    al_v = _angle(yd, xd)
    d_v = np.hypot(xd, yd)
    al_a = _angle(ydd, xdd)
    d_a = np.hypot(xdd, ydd)
    S = np.abs(np.sin(al_a - al_v))
    vmin_bar = np.maximum(prm.v_min, np.sqrt(da_prev * S / prm.kappa_max))
    cos2 = np.cos(al_v) ** 2
    kr = np.abs(road_at(scene, prm, x if x_prev is None else x_prev)[0])
    with np.errstate(divide="ignore"):
        vmax_bar = np.where(kr * cos2 > 0.0,
                            np.minimum(prm.v_max, np.sqrt(prm.c_max / np.maximum(kr * cos2, 1e-300))),
                            prm.v_max)
    d_v = np.minimum(np.maximum(d_v, vmin_bar), vmax_bar)        # clip_d_v
    kd = d_v ** 2 * prm.kappa_max
    with np.errstate(divide="ignore", invalid="ignore"):
        amax_bar = np.where(S * prm.a_max <= kd, prm.a_max, kd / S)
    d_a = np.minimum(np.maximum(d_a, 0.0), amax_bar)             # clip_d_a

    hvx, hvy = d_v * np.cos(al_v), d_v * np.sin(al_v)
    hax, hay = d_a * np.cos(al_a), d_a * np.sin(al_a)
    B = xi.shape[0]
    h = np.concatenate([hox.reshape(B, -1), hvx, hax, hoy.reshape(B, -1), hvy, hay], axis=1)
    parts = dict(d_o=d_o, al_o=al_o, d_v=d_v, al_v=al_v, d_a=d_a, al_a=al_a,
                 vmin_bar=vmin_bar, vmax_bar=vmax_bar, amax_bar=amax_bar,
                 hox=hox, hoy=hoy, hv=(hvx, hvy), ha=(hax, hay))
    return h, d_a, parts


def lane_vector(scene, prm, m):
    """e of Eq. (lane_reform): G xi <= e with G = [W; -W] on the y block
    (straight lanes; lane_vector_at for a road whose limits depend on x)."""
    ylb, yub = lane_bounds(scene, prm)
    return np.concatenate([np.full(m, yub), np.full(m, -ylb)])


def lane_vector_at(scene, prm, x):
    """e(xi) of Eq. (lane_reform) at the positions x (B, m) of an iterate:
    (B, 2m) = [y_ub(x), -y_lb(x)]."""
    _, ylb, yub = road_at(scene, prm, x)
    return np.concatenate([yub, -ylb], axis=1)


def slack_step(xi, G, e):
    """s = max(0, e - G xi), the minimiser of ||G xi - e + s||^2 over s >= 0;
    e is (2m,) or per sample (B, 2m)."""
    return np.maximum(0.0, np.atleast_2d(e) - xi @ G.T)


def xi_step(xi_bar, lam, h, s, ops, e, b_eq, rho):
    """Eq. (split_xy): minimise the augmented Lagrangian over xi with A xi = b."""
    F, G, A = ops
    nn = F.shape[1]
    H = np.eye(nn) + rho * (F.T @ F) + rho * (G.T @ G)
    rhs = xi_bar + lam + rho * (h @ F) + rho * ((np.atleast_2d(e) - s) @ G)
    return kkt_solve(H, A, rhs, b_eq)


def project(xi_bar, scene, prm, basis, iters: int | None = None, trace: bool = False, p=None):
    """Alg. 2 for every row of xi_bar; returns xi^K (and a per-iteration trace).
    With goal entries in p (prm.goal) the equality rows of Eq. split_xy carry
    each sample's b(p_j), so p (B, d_p) is required.

    The trace holds, per iteration, the mean over samples of
    ||F xi - h|| + ||G xi - e + s|| (the residual the multipliers drive to zero).
    """
    K = prm.inner_iters if iters is None else iters
    goal = getattr(prm, "goal", False)
    ops = projection_operators(basis, scene.n_obs, goal)
    F, G, A = ops
    if goal:
        if p is None:
            raise ValueError("goal entries: project needs p for b(p)")
        bx, by = equality_rhs(p, scene, prm)
        b_eq = np.concatenate([bx, by], axis=1)                         # (B, ne_x + ne_y)
    else:
        x0, y0, vx0, vy0, ax0, ay0 = np.asarray(scene.ego, dtype=np.float64)
        b_eq = [x0, vx0, ax0, y0, vy0, ay0]

    xi = np.array(xi_bar, dtype=np.float64, copy=True)
    lam = np.zeros_like(xi)
    x, _, _, _, xdd, ydd = kinematics(xi, basis)
    da = np.minimum(np.hypot(xdd, ydd), prm.a_max)
    e = lane_vector_at(scene, prm, x)                                   # e(^0 xi)
    h, da, _ = alpha_d_step(xi, scene, prm, basis, da, x)
    s = slack_step(xi, G, e)
    hist = []
    for _ in range(K):
        x_prev = x
        xi = xi_step(xi_bar, lam, h, s, ops, e, b_eq, prm.rho)           # split_xy with e(^k xi)
        x = kinematics(xi, basis)[0]
        h, da, _ = alpha_d_step(xi, scene, prm, basis, da, x_prev)      # split_alpha_o + clips
        e = lane_vector_at(scene, prm, x)                               # e(^{k+1} xi)
        s = slack_step(xi, G, e)                                        # update_slack
        rf = xi @ F.T - h
        rg = xi @ G.T - e + s
        lam = lam - 0.5 * prm.rho * (rf @ F) - 0.5 * prm.rho * (rg @ G)  # update_lagrange
        if trace:
            hist.append(float(np.mean(np.linalg.norm(rf, axis=1) + np.linalg.norm(rg, axis=1))))
    return (xi, hist) if trace else xi


# ----------------------------------------------------------------------------
# scoring (Alg. 1 line 9 and the upper-level cost of Sec. V-A)
# ----------------------------------------------------------------------------

def score(xi, scene, prm, basis):
    """r_j = sum over t (and obstacles) of max(0, g) for every row of Table I,
    and c_u = sum_t (sqrt(xd^2 + yd^2) - v_max)^2.  Returns (r, c_u), (B,) each.

    Curvature is taken as 0 where the speed is exactly 0.
    """
    m = basis[0].shape[0]
    x, y, xd, yd, xdd, ydd = kinematics(xi, basis)
    xo, yo, a, b = obstacle_trajectories(scene, m, prm.dt)
    dx = x[:, None, :] - xo[None]
    dy = y[:, None, :] - yo[None]
    coll = np.maximum(0.0, 1.0 - (dx / a[None]) ** 2 - (dy / b[None]) ** 2).sum(axis=(1, 2))
    speed = np.hypot(xd, yd)
    with np.errstate(divide="ignore", invalid="ignore"):
        kappa = np.where(speed > 0.0, (ydd * xd - xdd * yd) / speed ** 3, 0.0)
    kroad, ylb, yub = road_at(scene, prm, x)
    per_t = (np.maximum(0.0, speed - prm.v_max)
             + np.maximum(0.0, np.hypot(xdd, ydd) - prm.a_max)
             + np.maximum(0.0, np.abs(kappa) - prm.kappa_max)
             + np.maximum(0.0, xd ** 2 * np.abs(kroad) - prm.c_max)
             + np.maximum(0.0, y - yub) + np.maximum(0.0, ylb - y))
    r = coll + per_t.sum(axis=1)
    cu = ((speed - prm.v_max) ** 2).sum(axis=1)
    return r, cu


def solve(p, scene, prm, basis, iters: int | None = None):
    """Alg. 1 lines 6-9 for every p_j: Step 1, Step 2 (Alg. 2), residual and cost."""
    xb = step1(p, scene, prm, basis)
    xs = project(xb, scene, prm, basis, iters, p=p)
    r, cu = score(xs, scene, prm, basis)
    return xs, r, cu
