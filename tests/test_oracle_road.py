"""Pins of the oracle's road model (Table I's centripetal and lane-boundary
rows on a road given in the Frenet frame; Eqs. cent_bounds, clip_d_v,
lane_reform).

* road_at is piecewise-linear interpolation, checked against a direct
  evaluation written from the definition;
* a profile that repeats the constant road gives exactly the straight-road
  results;
* the velocity clip with road curvature lands h_v on the centripetal bound;
* the projection pulls trajectories into a narrowing road;
* the MPC advance keeps the road fixed in space while the frame moves."""
import numpy as np

from oracle import lower, mpc
from oracle.basis import bernstein
from paper_2212_02224_gb300 import scenegen as sg


def _direct(knots, x):
    """Piecewise-linear value of knot columns 1..3 at x, held beyond the ends."""
    s = knots[:, 0]
    out = np.empty((len(x), 3))
    for i, xv in enumerate(x):
        if xv <= s[0]:
            out[i] = knots[0, 1:]
        elif xv >= s[-1]:
            out[i] = knots[-1, 1:]
        else:
            k = max(j for j in range(len(s)) if s[j] <= xv)
            w = (xv - s[k]) / (s[k + 1] - s[k])
            out[i] = (1 - w) * knots[k, 1:] + w * knots[k + 1, 1:]
    return out


def test_road_at_is_piecewise_linear():
    prm = sg.Params(lane_margin=0.7)
    sc = sg.make_scene(1, n_lanes=3, n_obs=0)
    sc.road = sg.curved_road(3, kappa=0.02)
    sc.road_origin = 12.5
    x = np.linspace(-30.0, 220.0, 501)
    kap, lb, ub = lower.road_at(sc, prm, x)
    ref = _direct(sc.road, x + 12.5)
    np.testing.assert_allclose(kap, ref[:, 0], atol=1e-15)
    np.testing.assert_allclose(lb, ref[:, 1] + 0.7, atol=1e-12)
    np.testing.assert_allclose(ub, ref[:, 2] - 0.7, atol=1e-12)


def test_constant_profile_reproduces_the_straight_road():
    prm, sc, _ = sg.workload(0, inner_iters=20)
    sc.kappa_road = 0.004
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    p = sg.make_samples(4, sc, 12, prm.n_seg)
    ref = lower.solve(p, sc, prm, basis)
    w = sc.n_lanes * sc.lane_width
    sc.road = np.array([[-50.0, 0.004, 0.0, w], [80.0, 0.004, 0.0, w], [300.0, 0.004, 0.0, w]])
    got = lower.solve(p, sc, prm, basis)
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a, b)


def test_velocity_clip_meets_the_centripetal_bound():
    """Eq. (cent_bounds): d_v^2 cos^2(alpha_v) |kappa| <= c_max after the clip,
    with kappa taken at the previous iterate's positions."""
    prm = sg.Params(m=60, c_max=2.0)
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    sc = sg.make_scene(2, n_lanes=3, n_obs=0)
    sc.road = sg.curved_road(3, kappa=0.03, bend=(0.0, 200.0), narrow_at=None)
    p = sg.make_samples(6, sc, 16, 1, v_range=(15.0, 25.0))
    xi = lower.step1(p, sc, prm, basis)
    x, _, xd, yd, xdd, ydd = lower.kinematics(xi, basis)
    x_prev = x - 3.0                      # any earlier positions
    da = np.minimum(np.hypot(xdd, ydd), prm.a_max)
    _, _, parts = lower.alpha_d_step(xi, sc, prm, basis, da, x_prev)
    kap = np.abs(lower.road_at(sc, prm, x_prev)[0])
    hvx = parts["hv"][0]
    lhs = hvx ** 2 * kap
    assert (lhs <= prm.c_max * (1 + 1e-12)).all()
    bound = np.sqrt(prm.c_max / np.maximum(kap * np.cos(parts["al_v"]) ** 2, 1e-300))
    active = parts["d_v"] < np.hypot(xd, yd) - 1e-9
    np.testing.assert_allclose(parts["d_v"][active], np.minimum(prm.v_max, bound)[active],
                               rtol=1e-12)
    assert active.any()


def test_projection_follows_a_narrowing_road():
    """Samples that aim at the top lane of a road that loses it: the Step-1
    trajectories leave the road, the projected ones stay within the limits
    up to a small residual."""
    prm = sg.Params(m=100, inner_iters=200)
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    sc = sg.make_scene(3, n_lanes=3, n_obs=0, ego_lane=2)
    sc.road = sg.curved_road(3, kappa=0.0, narrow_at=40.0)
    p = np.array([[sc.lane_centres()[2], v] for v in (12.0, 16.0, 20.0)])
    xb = lower.step1(p, sc, prm, basis)
    xs = lower.project(xb, sc, prm, basis)

    def excess(xi):
        x, y = lower.kinematics(xi, basis)[:2]
        _, lb, ub = lower.road_at(sc, prm, x)
        return np.maximum(0.0, y - ub).max(), np.maximum(0.0, lb - y).max()

    before, after = excess(xb), excess(xs)
    assert before[0] > 1.0
    assert after[0] < 0.05 and after[1] < 0.05


def test_advance_keeps_the_road_fixed():
    prm, sc, _ = sg.workload(0)
    sc.road = sg.curved_road(sc.n_lanes, kappa=0.01)
    basis = bernstein(prm.m, prm.n_coef, prm.dt)
    p = sg.make_samples(8, sc, 1, prm.n_seg)
    xi = lower.step1(p, sc, prm, basis)[0]
    nxt = mpc.advance(sc, xi, prm, steps=5, basis=basis)
    x5 = lower.kinematics(xi[None], basis)[0][0, 5]
    assert nxt.road_origin == sc.road_origin + x5
    q = np.linspace(-10.0, 150.0, 50)
    for a, b in zip(lower.road_at(nxt, prm, q), lower.road_at(sc, prm, q + x5)):
        np.testing.assert_allclose(a, b, rtol=1e-14, atol=1e-14)
