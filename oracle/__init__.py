"""Plain FP64 CPU oracle for s-step Orthomin(k) and s-step GMRES(m).

TEST INFRASTRUCTURE ONLY. This package is the independent, slow, obviously
correct restatement of Chronopoulos & Kim, "s-Step Orthomin and GMRES
implemented on parallel computers" (1990), written in numpy float64. Only the
test suite, the smoke check in __graft_entry__ and the CPU-baseline leg of
bench.py may import it. The library (paper_2001_04886_gb300) never imports it,
and it imports nothing from the library. The seeded input generators are the
only code both sides use, and they hold none of the method's arithmetic.

Modules
  stencil  - the operator A of Sec. 5 / Sec. 1 (5- and 7-point convection-
             diffusion stencils with homogeneous Dirichlet boundaries).
  krylov   - Algorithm 2.1 (Orthomin(k)) and Algorithm 2.2 (GMRES(m)), plus the
             Givens least-squares of eq. 2.
  sstep    - Algorithm 3.1 (s-step Orthomin(k)) and Algorithms 4.1/4.2
             (s-step Arnoldi / s-step GMRES), with their block primitives.
  dense    - dense matrices of tiny operators and a direct solve, used only to
             pin the iterative solvers by brute force.

Parity status: every function here is pinned by a -m "not gpu" test against
closed forms, brute force or special cases that reduce to other algorithms;
see tests/test_oracle_*.py. No function is "parity unpinned".
"""

STATUS_OK = 0
STATUS_NOT_CONVERGED = 1
STATUS_BREAKDOWN = -4
