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
The exact values of the Alg. 2 iterates beyond those invariants (a
non-convex alternating minimisation) have no independent closed form; the
convex special case (lane bounds only) is pinned against a general QP solve.
Status of ``lower.solve`` on a general scene: parity unpinned for the exact
iterate values (only the invariants above and the oracle-vs-GPU agreement
hold them); every other function is pinned.
"""
