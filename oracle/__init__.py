"""FP64 CPU oracle for the multi-patch isogeometric multigrid solver (Hofer & Takacs,
"A parallel multigrid solver for multi-patch Isogeometric Analysis").

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, readable restatement of the
method in NumPy/SciPy, used to check the CUDA library.  Only the tests, the smoke check
and the CPU-baseline leg of the benchmark may import it; the library never does, and it
never imports the library.  It shares no code with the CUDA path: the only common module
is `workloads`, which holds the seeded problem descriptions and no arithmetic of the
method.

Modules (each function cites the passage it follows):
  bspline    univariate spline spaces S_{p,h} (Sec. 2), Gauss quadrature, 1D mass and
             stiffness matrices, knot insertion (Sec. 3, the canonical embedding P_l)
  patch      multilinear geometry maps G_k and the patch forms a_k (Eq. model:bil)
  multipatch fully matching multi-patch space V_l (Eq. vh), dof numbering, Dirichlet
             elimination, pieces of the additive Schwarz smoother (Eq. additive)
  smoother   patch-interior subspace-corrected mass smoother, edge/face/vertex smoothers
             (Sec. 3 list of local smoothers)
  solver     grid hierarchy, the multigrid cycle (Algorithm 1), PCG, dense direct solve

Parity status: every function is pinned by tests in tests/test_oracle_*.py against
closed forms, invariants, brute force or the dof counts printed for the Fichera corner
(Table II); the subspace-corrected mass smoother follows a reading of a reference that
is not part of the paper text (see the module docstring of `smoother`), so its
*definition* is a reading, while its implementation is pinned by the identities listed
there.
"""
