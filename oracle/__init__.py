"""CPU FP64 oracle for the adAFAC multigrid cycle (Murray & Weinzierl,
"Stabilised Asynchronous Fast Adaptive Composite Multigrid using Additive
Damping", arXiv:1903.10367).

THIS PACKAGE IS TEST INFRASTRUCTURE.  It is a plain, slow, obviously correct
restatement of what the paper's method computes, written from the paper in
numpy/scipy FP64.  Only the test-suite, the ``smoke()`` entry of
``__graft_entry__`` and the ``cpu_baseline``/reference leg of ``bench.py`` may
import it.  The CUDA library never calls into it and shares no code with it
(they share only the seeded input generators in ``workloads``).

Modules
-------
fem       d-linear finite elements on a 3:1 spacetree level (Eq. 1, Sec. 2.1)
transfer  d-linear and BoxMG prolongation, restriction R = P^T, Galerkin
          coarse operators (Sec. 2.2, 2.4)
cycle     smoothed restriction R~ (Sec. 3.2), the adAFAC-Jac cycle (Alg. 1,
          Eq. 9) in correction-scheme and FAS/HTMG form (Eq. 4), adAFAC-PI
          (Alg. 2), plain additive multigrid (Eq. 2) with optional exponential
          damping, and the normalised residual (Eq. 10)
adaptive  the same cycles on adaptive spacetrees with hanging vertices, over
          the hierarchical generating system of all levels' pagodas
          (Sec. 2.1, 2.3)

Every function is pinned by ``tests/test_oracle_*.py`` against facts that do
not come from the oracle itself (closed forms, the paper's printed stencil,
brute-force quadrature and dense linear algebra on tiny grids, a direct solve,
the O(h^2) error of a manufactured solution).
"""
