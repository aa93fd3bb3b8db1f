"""FP64 CPU oracle for the H1-regularized Gauss-Newton linear solve.

TEST INFRASTRUCTURE ONLY. Only the test suite, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / reference legs of ``bench.py`` may import, call, link or
execute anything in this package. The product path (the CUDA library and its
Python binding) never routes through it and shares no code with it.

What it computes, written from the paper's definitions and kept deliberately
plain (no blocking, fusion or reordering beyond what the definitions state):

* ``discretization``: the regularization operator K + M assembled as sparse
  matrices element by element (bilinear Q1 on vertex grids in 2D; cell-centred
  finite volumes in 3D, i.e. the lowest-order Raviart-Thomas Schur complement
  D diag(Q)^-1 D^T of Sec. 2.3 on a Cartesian grid).
* ``multigrid``: the Laplace preconditioner L^-1 as one symmetric V-cycle
  (Chebyshev-Jacobi smoothing, linear/trilinear transfer, dense coarsest solve),
  the operator written with sparse matrices and recursion.
* ``woodbury``: the capacitance matrix C = I + alpha^-1 J H, H = L^-1 J^T
  (Algorithm "MINRES with the Laplace-Woodbury preconditioner", lines H/C/chol)
  and the Sherman-Morrison-Woodbury preconditioner apply (Sec. 3.2), the dense
  direct Woodbury solve of Sec. 3.1, and PCG with the Euclidean stopping rule.
* ``ert``: the ERT forward model of Sec. 4.1 on a cell-centred finite-volume
  grid (harmonic-mean face conductances, Dirichlet ghosts, unit point
  currents), its measurements (Eqs. 4.3, 4.5) and Jacobian (Eq. 4.4), by
  sparse LU solves.
* ``ccg``: a plain C + OpenMP operator apply and unpreconditioned CG on the
  assembled CSR operator plus the two dense J products (the timed CPU
  baseline).

Pins (tests marked ``not gpu``) tie each part to something other than itself:
closed-form cosine eigenpairs of the grid operators, Chebyshev error
polynomials, the Woodbury identity with an exact Laplace inverse (one PCG
iteration), brute-force dense solves, symmetry, and the m = 0 / m = 1 special
cases.
"""
