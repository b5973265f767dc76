"""FP64 CPU oracle of the bi-level planner's lower-level optimizer and Alg. 1.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
reference that the CUDA path is checked against.  Only the test-suite, the
smoke check in ``__graft_entry__`` and the CPU-baseline leg of ``bench.py``
may import it; the product library never does, and this package imports
nothing from the product.

Everything is float64 numpy, batched over samples the way the paper batches
them (Eq. over_3), and follows the paper's steps in its order and notation:

* ``basis``   -- the polynomial trajectory parametrisation, Eq. (param).
* ``lower``   -- Step 1 (the equality-constrained QP of Alg. 1, solved via the
  KKT system of Eq. over_2), the batch projection of Alg. 2
  (Eqs. split_xy .. update_lagrange) and the residual / driving-cost scoring
  (Alg. 1 line 9, Sec. V-A upper-level cost).
* ``upper``   -- Alg. 1: sampling, ConstraintEliteSet / EliteSet selection and
  the distribution update of Eqs. (mean_update, cov_update, s_formula), with
  a Philox4x32-10 counter-based generator (Salmon et al., SC'11) so that the
  CUDA side can draw the same numbers from the same published definition.

Readings of garbled or unstated parts of the paper (sign of the PD tracking
terms, the slack and multiplier updates, the curvature-derived bounds, tie
breaks, the first-iteration distribution) are stated at each function.

Pinning: every function here is pinned by the not-gpu tests against closed
forms, invariants of the constraint sets, library routines or brute force.
The Alg. 2 iterates (a non-convex alternating minimisation) have no closed
form; beyond the invariants (A xi = b every iteration, the fixed point at a
feasible xi_bar, the convex lane case against a general QP solve) the
iteration map is pinned by a second statement of Alg. 2 written row by row
from the paper (its own assembly, projections and a null-space xi-step),
which fixes the multiplier step rho/2 and the lagged curvature of the
velocity clip.  Where the paper is garbled both statements take the same
reading (stated at each function); a reading is a choice, not a pin.
"""
