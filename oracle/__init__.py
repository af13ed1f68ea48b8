"""Plain FP64 CPU oracle for piece-wise-constant-tested isogeometric analysis.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports this
module; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` may use it.  It shares no code, tables or
constants with the CUDA path: it evaluates B-splines with its own Cox--de Boor
recursion, integrates with Gauss--Legendre rules from numpy, assembles the
Galerkin and piece-wise-constant (PW) systems entry by entry, and solves them
with pivoted dense LU (numpy/LAPACK).

Modules
  bspline     knot vectors, Cox--de Boor values and derivatives   (Sec. 2, Eq. (2))
  quadrature  Gauss rules, Greville abscissae, PW test cells       (Sec. 2, Sec. 4.1)
  systems     1D Galerkin / PW matrices, Dirichlet rows            (Sec. 2, Sec. 4.3)
  tensor      d-D quadrature-grid evaluation and testing,
              tensor-product systems, ADS Kronecker solve          (Sec. 3, Sec. 4.1)
  heat        explicit Euler steps (one L2 projection per step)    (Sec. 4.2, Eq. (6))
  poisson     1D Poisson with zero Dirichlet rows                  (Sec. 4.3, Eq. (7))

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
library routines, invariants or brute force (see those tests).
"""
