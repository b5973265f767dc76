"""Checks of the reduced-precision error model (tests/error_model.py) on the
CPU: no rounding gives no deviation, a feasible Step-1 solution (no active
projection) is left exactly where it is, and the deviation is first order in
the unit roundoff."""
import numpy as np

import error_model as em
from paper_2212_02224_gb300 import scenegen as sg


def _case(n_obs=3, B=6, K=12):
    prm = sg.Params(m=40, n_coef=11, inner_iters=K)
    sc = sg.make_scene(31, n_lanes=3, n_obs=n_obs, obs_x=(10.0, 40.0))
    p = sg.make_samples(4, sc, B, 1)
    return prm, sc, p


def test_no_rounding_no_deviation():
    prm, sc, p = _case()
    d_pos, d_r, d_cu = em.predicted_deviation(prm, sc, p, 0.0, draws=2)
    assert d_pos.max() <= 1e-12 and d_r.max() <= 1e-12 and d_cu.max() <= 1e-12


def test_inactive_rows_carry_no_error():
    """No obstacles and loose bounds: every projection is inactive, the kernel's
    residual rows are exactly zero, and the modelled deviation is zero up to
    the float64 rounding of the oracle's own projection (atan2 / cos / sin)."""
    prm, sc, p = _case(n_obs=0)
    prm.v_max, prm.a_max, prm.kappa_max, prm.v_min = 80.0, 80.0, 1e3, 0.0
    sc.n_lanes = 8
    d_pos, _, _ = em.predicted_deviation(prm, sc, p, 2.0 ** -8, draws=2)
    assert d_pos.max() <= 1e-9


def test_deviation_is_first_order_in_u():
    prm, sc, p = _case()
    a = em.predicted_deviation(prm, sc, p, 1e-9, draws=1, seed=3)[0]
    b = em.predicted_deviation(prm, sc, p, 2e-9, draws=1, seed=3)[0]
    assert a.max() > 0
    ratio = b.max() / a.max()
    assert 1.8 <= ratio <= 2.2, ratio
