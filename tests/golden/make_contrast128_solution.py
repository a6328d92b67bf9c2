"""Write tests/golden/contrast128_solution.txt: samples of the solution of
A u = f for the 128^3 benchmark problem, computed by the oracle alone.

Problem (the benchmark's own seeded inputs): n = 128 (N = 2,097,152), zero
Dirichlet boundary, a = 10^U(-1,1) iid per grid point (seed 20260103), b = 0.1,
f = one N(0,1) grid function (seed 20260104); A is the seven-point operator of
§2.4 (oracle.stencil.assemble).  The solution is computed by the oracle's
Jacobi-preconditioned conjugate gradients to ||f - A u|| <= 1e-14 ||f||
(oracle.krylov.cg_jacobi), no HIF involved.

Stored: the sizes and seeds, the residual reached, ||u||_2, ||u||_inf, the
inner products <u, g_k> with four seeded N(0,1) vectors g_k (seeds 20260300 +
k), and u at 1024 seeded sample points (seed 20260400).  Run:

    python tests/golden/make_contrast128_solution.py
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import krylov, stencil  # noqa: E402
from paper_1607_00346_gb300 import inputs  # noqa: E402

N_GRID = 128
SEED_A = inputs.SEED_BASE + 2
SEED_F = SEED_A + 1
B = 0.1
SEED_G = 20260300
SEED_SAMPLES = 20260400
N_SAMPLES = 1024
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "contrast128_solution.txt")


def sample_points(N: int) -> np.ndarray:
    return np.sort(inputs.rng(SEED_SAMPLES).choice(N, size=N_SAMPLES, replace=False))


def main():
    n = N_GRID
    N = n ** 3
    a = inputs.coeff_log_uniform(n, -1.0, 1.0, SEED_A)
    f = inputs.normal_rhs(n, 1, SEED_F)[0]
    A = stencil.assemble(a, B, n)
    t0 = time.time()
    u, its, rel = krylov.cg_jacobi(A, f, tol=1e-14, max_iter=200000)
    dt = time.time() - t0
    idx = sample_points(N)
    with open(OUT, "w") as fh:
        fh.write("# solution samples of A u = f, 128^3 benchmark problem (oracle Jacobi-CG)\n")
        fh.write("# written by tests/golden/make_contrast128_solution.py\n")
        fh.write(f"n {n}\nseed_a {SEED_A}\nseed_f {SEED_F}\nb {B!r}\n")
        fh.write(f"cg_iterations {its}\nrelres {rel:.6e}\n")
        fh.write(f"norm2 {np.linalg.norm(u):.17e}\nnorminf {np.abs(u).max():.17e}\n")
        for k in range(4):
            g = inputs.normal_rhs(n, 1, SEED_G + k)[0]
            fh.write(f"dot {SEED_G + k} {float(u @ g):.17e}\n")
        fh.write(f"samples {N_SAMPLES} seed {SEED_SAMPLES}\n")
        for i in idx:
            fh.write(f"{int(i)} {u[i]:.17e}\n")
    print(f"cg: {its} iterations, relres {rel:.3e}, {dt:.1f} s -> {OUT}")


if __name__ == "__main__":
    main()
