"""Plain, slow, FP64 CPU oracle of the hierarchical interpolative factorization.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute anything in this package: only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.
It shares no code with the CUDA path (different language, different data
structures) and takes every input as a plain numpy array.

Method: Li & Ying, "Distributed-memory Hierarchical Interpolative
Factorization" (arXiv:1607.00346).  The oracle follows the sequential HIF of
§2.4 step by step, with the readings listed per module:

* ``stencil``  -- the seven-point discretisation of -div(a grad u) + b u (§2.4,
  seven-point stencil equation), zero Dirichlet boundary.
* ``geometry`` -- cells, faces, edges and vertices of §2.1 on the Dirichlet
  grid.
* ``cpqr``     -- column-pivoted Householder QR and the interpolative
  decomposition of §2.3.
* ``hif``      -- sparse elimination (§2.2), skeletonization (§2.3), the level
  loop and root factorization (§2.4), and the application of F^{-1}.
* ``krylov``   -- the solve error e_s of Table 2, a power-iteration estimate
  of ||I - F^{-1} A||, and PCG with F^{-1} as preconditioner.

Every function is pinned by tests/test_oracle_*.py against closed forms,
LAPACK, dense direct solves and algebraic identities; see those tests.
"""
