"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of one oracle function (a dropped term,
a flipped sign, a swapped index or operand, a missing factor), patches it into
the oracle module, and runs the pins that cover that function: at least one of
them must fail.  The mistakes are planted in the oracle on the CPU only."""
import inspect
import textwrap

import pytest

import test_oracle_alg2_rowwise as ta
import test_oracle_basis as tb
import test_oracle_goal as tg
import test_oracle_lower as tl
import test_oracle_qp_layer as tq
import test_oracle_road as tr
import test_oracle_upper as tu
from oracle import basis as obasis
from oracle import lower, upper

# (module, function, snippet, replacement, pins)
MUTATIONS = [
    ("basis: derivative not scaled by 1/t_f", obasis, "bernstein",
     "return W, dW / tf, ddW / tf ** 2", "return W, dW, ddW / tf ** 2",
     [lambda: tb.test_finite_differences()]),
    ("Step 1: smoothness term dropped", lower, "step1_cost_matrices",
     "Qx = 2.0 * (Wdd.T @ Wdd + Lx.T @ Lx)", "Qx = 2.0 * (Lx.T @ Lx)",
     [lambda: tl.test_step1_is_constrained_minimiser(1), tl.test_step1_null_space_method_agrees]),
    ("Step 1: tracking gain sign flipped", lower, "step1",
     "qx = -2.0 * prm.kp_lon * (vd @ Lx)", "qx = 2.0 * prm.kp_lon * (vd @ Lx)",
     [tl.test_step1_closed_form_steady_state, lambda: tl.test_step1_is_constrained_minimiser(1)]),
    ("Step 1: velocity row taken twice in A", lower, "initial_rows",
     "np.stack([W[0], Wd[0], Wdd[0]])", "np.stack([W[0], Wd[0], Wd[0]])",
     [lambda: tl.test_step1_is_constrained_minimiser(1), tl.test_step1_closed_form_steady_state]),
    ("set-points: y_d and v_d halves swapped", lower, "setpoint_vectors",
     "return p[:, :n_seg][:, seg_of_t], p[:, n_seg:2 * n_seg][:, seg_of_t]",
     "return p[:, n_seg:2 * n_seg][:, seg_of_t], p[:, :n_seg][:, seg_of_t]",
     [tl.test_setpoint_segments]),
    ("obstacle h_y with a instead of b", lower, "alpha_d_step",
     "hoy = yo[None] + b[None] * d_o * np.sin(al_o)", "hoy = yo[None] + a[None] * d_o * np.sin(al_o)",
     [tl.test_obstacle_projection_lands_on_constraint_set]),
    ("obstacle clip min instead of max", lower, "alpha_d_step",
     "d_o = np.maximum(1.0, d_o)", "d_o = np.minimum(1.0, d_o)",
     [tl.test_obstacle_projection_lands_on_constraint_set]),
    ("v_min-bar without kappa_max", lower, "alpha_d_step",
     "np.sqrt(da_prev * S / prm.kappa_max)", "np.sqrt(da_prev * S)",
     [tl.test_velocity_acceleration_projection_invariants, tl.test_vmin_bar_binds_at_low_speed]),
    ("acceleration clip lost", lower, "alpha_d_step",
     "d_a = np.minimum(np.maximum(d_a, 0.0), amax_bar)", "d_a = np.maximum(d_a, 0.0)",
     [tl.test_velocity_acceleration_projection_invariants]),
    ("slack sign garbled", lower, "slack_step",
     "np.maximum(0.0, np.atleast_2d(e) - xi @ G.T)", "np.maximum(0.0, xi @ G.T - np.atleast_2d(e))",
     [tl.test_slack_nonnegative_and_exact_when_feasible]),
    ("xi-step without the multipliers", lower, "xi_step",
     "rhs = xi_bar + lam + rho", "rhs = xi_bar + rho",
     [tl.test_xi_step_minimises_augmented_lagrangian]),
    ("multiplier update sign flipped", lower, "project",
     "lam = lam - 0.5 * prm.rho * (rf @ F) - 0.5 * prm.rho * (rg @ G)",
     "lam = lam + 0.5 * prm.rho * (rf @ F) + 0.5 * prm.rho * (rg @ G)",
     [tl.test_projection_reduces_residual_on_static_obstacles, tl.test_convex_lane_case_limit]),
    ("multiplier step rho instead of the printed rho/2", lower, "project",
     "lam = lam - 0.5 * prm.rho * (rf @ F) - 0.5 * prm.rho * (rg @ G)",
     "lam = lam - 1.0 * prm.rho * (rf @ F) - 1.0 * prm.rho * (rg @ G)",
     [lambda: ta.test_project_matches_rowwise_restatement(2)]),
    ("road curvature of the velocity clip at the current iterate", lower, "project",
     "h, da, _ = alpha_d_step(xi, scene, prm, basis, da, x_prev)",
     "h, da, _ = alpha_d_step(xi, scene, prm, basis, da, x)",
     [lambda: ta.test_project_matches_rowwise_restatement(2)]),
    ("goal: x_f and y_f swapped in b(p)", lower, "equality_rhs",
     "bx = np.column_stack([bx, p[:, 2 * ns]])", "bx = np.column_stack([bx, p[:, 2 * ns + 1]])",
     [tg.test_goal_cruise_closed_form, tg.test_goal_rows_hold_every_iteration]),
    ("goal: final lateral acceleration row instead of velocity", lower, "equality_rows",
     "np.vstack([A0, W[-1], Wd[-1]])", "np.vstack([A0, W[-1], Wdd[-1]])",
     [tg.test_goal_rows_hold_every_iteration, tg.test_goal_step1_null_space_method_agrees]),
    ("goal prior: x_f without the horizon length", upper, "draw_initial",
     "float(scene.ego[0]) + (prm.m - 1) * prm.dt * speed(u[:, 2 * ns])",
     "float(scene.ego[0]) + speed(u[:, 2 * ns])",
     [tg.test_goal_initial_draws_and_moments]),
    ("goal VJP: x_f and y_f gradients swapped", lower, "step1_layer_vjp",
     "grad_p[:, 2 * prm.n_seg + axis] = w[:, 3]", "grad_p[:, 2 * prm.n_seg + 1 - axis] = w[:, 3]",
     [tg.test_goal_layer_vjp_matches_central_differences]),
    ("score: lane rows swapped", lower, "score",
     "np.maximum(0.0, y - yub) + np.maximum(0.0, ylb - y)",
     "np.maximum(0.0, y - ylb) + np.maximum(0.0, yub - y)",
     [tl.test_score_lane_and_collision_rows, tl.test_fixed_point_when_feasible]),
    ("road: lane margin not applied", lower, "road_at",
     "ylb = np.interp(x, sk, road[:, 2]) + prm.lane_margin", "ylb = np.interp(x, sk, road[:, 2])",
     [tr.test_road_at_is_piecewise_linear]),
    ("layer VJP: factor 2k dropped", lower, "step1_layer_vjp",
     "ds = 2.0 * k * (u @ L.T)", "ds = (u @ L.T)",
     [lambda: tq.test_vjp_matches_central_differences(1, 11), tq.test_dot_product_identity]),
    ("elite weights grow with cost", upper, "update_distribution",
     "s = np.exp(-(cost_elite - cost_elite.min()) / prm.gamma)",
     "s = np.exp((cost_elite - cost_elite.min()) / prm.gamma)",
     [tu.test_update_distribution_weights_follow_costs]),
    ("ties broken by the higher index", upper, "select_lowest",
     "order = np.lexsort((idx, k))", "order = np.lexsort((-idx, k))",
     [tu.test_select_lowest_matches_sorted_with_ties]),
]


def _mutant(module, fname, old, new):
    src = textwrap.dedent(inspect.getsource(getattr(module, fname)))
    assert src.count(old) >= 1, f"snippet not found in {fname}: {old}"
    ns = dict(module.__dict__)
    exec(compile(src.replace(old, new, 1), f"<mutant of {fname}>", "exec"), ns)
    return ns[fname]


@pytest.mark.parametrize("case", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(case, monkeypatch):
    _, module, fname, old, new, pins = case
    monkeypatch.setattr(module, fname, _mutant(module, fname, old, new))
    if module is obasis:
        monkeypatch.setattr(tb, "bernstein", getattr(module, fname))
    failed = 0
    for pin in pins:
        try:
            pin()
        except Exception:      # a failed check, or the oracle breaking down
            failed += 1
    assert failed >= 1, "no pin caught the planted mistake"


def test_unmutated_pins_pass():
    """The same pins pass on the oracle as committed."""
    for case in MUTATIONS:
        for pin in case[5]:
            pin()
