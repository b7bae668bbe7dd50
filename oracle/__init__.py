"""CPU oracle for the hybrid multigrid DG method of Bastian, Mueller, Muething,
Piatkowski (arXiv 1805.11930).

TEST INFRASTRUCTURE ONLY.  Nothing in the library calls this package; only the
tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl
reference`` legs of ``bench.py`` may import it.  It shares no code with the
CUDA path: it assembles the DG matrix explicitly from the bilinear form by
direct quadrature (Sec. 2.1, eq. bilinear_form_split), stores it in block-CSR
form, inverts the diagonal blocks with dense LU, and builds the Q1 coarse
space, aggregation AMG, V-cycle (Algorithm 1) and Krylov solvers on top of
that matrix.  Everything is float64 (the paper's precision).

Modules
-------
quadrature   Gauss-Legendre / Gauss-Lobatto rules and 1D Lagrange bases.
dg           mesh, coefficients, explicit assembly of A and of the RHS.
transfer     Q1 prolongation P, restriction R = P^T, Q1 re-discretisation.
amg          aggregation AMG (structured 2x2x2 aggregates, Galerkin levels).
solvers      block-Jacobi (exact and inexact), V-cycle, CG, FCG, FGMRES.
"""
