"""Plain, slow FP64 CPU oracle for the matrix-free phase-field fracture solver.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU-baseline legs of
bench.py may import, call, link or execute anything under oracle/.  The oracle shares no code
with the CUDA library and never imports it; the two meet only through the seeded input
generators of paper_1902_08112_gb300.workloads, which hold none of the method's arithmetic.

Layers (each cites the passage it follows):
  fem.py        element-by-element assembly of the Jacobian, residual, energy, lumped mass
                (C core in pff_oracle.c)
  multigrid.py  transfers, level state restriction, Chebyshev-Jacobi, eigenvalue estimate,
                coarse solver, V-cycle
  krylov.py     flexible GMRES
  pdas.py       one primal-dual active-set step (Algorithm 1)
  rng.py        SplitMix64 counter-based generator (CG start vector)

Parity status: every function is pinned by tests/test_oracle_*.py except where its docstring
says "parity unpinned" (iteration counts of the solver stack are pinned only by ranges).
"""
from . import fem, multigrid, krylov, rng  # noqa: F401
