"""CPU oracle for the hybrid factorization (arXiv 2208.01907).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The library's
product path never calls it and shares no code with it.

Plain, slow, readable numpy.  Each function cites the passage of the paper it
restates.  Decisions that the paper makes in the lower precision (pivot choice
and threshold postponing, Alg. 1 step 1) are taken in float32; everything the
paper computes in the higher precision is float64.

Parity status per function (what pins it is listed in tests/test_oracle_*.py):
  scale_matrix            pinned (closed form, Sec. 2)
  nested_dissection       pinned (separator property, Fig. 1 block pattern)
  threshold_factorize     pinned (Eq. 1 reconstruction in LDL^T and LDU form, tiny hand cases,
                                  tau limits, brute-force Schur complements, the row-sign identity)
  precond_apply           pinned (exact inverse of the recorded factor, symmetric and unsymmetric)
  block_gcr               pinned (invariants of Sec. 3.4-3.5, direct solve)
  gcr_single              pinned (Krylov minimal residual with Q = I, equals block_gcr on one column)
  iterative_refinement    pinned (closed form r_n = (I - A Q^-1)^n r_0 of Sec. 3.3)
  schur_direct            pinned (dense brute-force inverse, Eq. 2)
  bunch_kaufman           pinned (reconstruction, scipy/LAPACK sytrf comparison)
  bunch_parlett           pinned (reconstruction, inertia, step-by-step brute-force choice, rank)
  lu_complete             pinned (reconstruction, step-by-step brute-force choice, rank revealing)
  lu_pseudo_solve         pinned (dense solve, consistent singular systems)
  kernel_dimension        pinned (dense SVD rank on small systems)
  hybrid_solve            pinned (backward error, exact solution on small systems, LDU form)
  s22_noise               pinned (the Schur change from a perturbed X12)
  relative_residual,
  backward_error          pinned (hand-worked 2x2 case)
  adjoint_gradient        pinned (central finite differences)
"""
from .hybrid import *  # noqa: F401,F403
