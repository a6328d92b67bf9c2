"""Accuracy metrics and the preconditioned solve (oracle; test infrastructure only).

* e_s = ||(I - F^{-1} A) x|| / ||x|| with x Gaussian (Table 2, "relative
  error for solving").
* power-iteration estimate of the spectral radius of I - F^{-1} A, i.e.
  max |1 - lambda| over the eigenvalues of F^{-1} A (both SPD, so the
  eigenvalues are real and positive).
* conjugate gradients on A u = f with the diagonal of A as preconditioner:
  no HIF at all, a plain route to the solution of the discrete problem
  (eq. 1 with the stencil of §2.4; A is SPD) at sizes where the HIF oracle
  is too slow;
* PCG with F^{-1} as preconditioner.  The paper runs GMRES to 1e-12 (Table 2);
  F^{-1} = W D^{-1} W^T is SPD when D > 0, so conjugate gradients apply.  The
  Polak-Ribiere form of beta is used so that a slightly non-symmetric
  (rounded) preconditioner is tolerated.  Stop when ||r||_2 / ||f||_2 <= tol.
"""
from __future__ import annotations

import numpy as np

from .hif import Factor, hif_apply


def solve_error(A, fac: Factor, x: np.ndarray) -> float:
    x = np.asarray(x, dtype=np.float64)
    r = x - hif_apply(fac, A @ x)
    return float(np.linalg.norm(r) / np.linalg.norm(x))


def power_norm(A, fac: Factor, seed_vec: np.ndarray, iters: int = 40) -> float:
    """Estimate max |1 - lambda(F^{-1} A)| by power iteration on I - F^{-1} A."""
    v = np.asarray(seed_vec, dtype=np.float64).copy()
    v /= np.linalg.norm(v)
    est = 0.0
    for _ in range(iters):
        w = v - hif_apply(fac, A @ v)
        nw = np.linalg.norm(w)
        if nw == 0.0:
            return 0.0
        est = nw
        v = w / nw
    return float(est)


def pcg(A, fac: Factor, f: np.ndarray, tol: float = 1e-10, max_iter: int = 200,
        u0: np.ndarray | None = None):
    """Solve A u = f; returns (u, iterations, relative residual history)."""
    f = np.asarray(f, dtype=np.float64)
    u = np.zeros_like(f) if u0 is None else np.array(u0, dtype=np.float64)
    r = f - A @ u
    fn = np.linalg.norm(f)
    hist = [np.linalg.norm(r) / fn]
    if hist[-1] <= tol:
        return u, 0, hist
    z = hif_apply(fac, r)
    p = z.copy()
    rz = r @ z
    for it in range(1, max_iter + 1):
        Ap = A @ p
        alpha = rz / (p @ Ap)
        u += alpha * p
        r_old = r
        r = r - alpha * Ap
        hist.append(np.linalg.norm(r) / fn)
        if hist[-1] <= tol:
            return u, it, hist
        z = hif_apply(fac, r)
        rz_new = r @ z
        beta = (z @ (r - r_old)) / rz        # Polak-Ribiere
        rz = rz_new
        p = z + beta * p
    return u, max_iter, hist


def cg_jacobi(A, f: np.ndarray, tol: float = 1e-14, max_iter: int = 100000):
    """Solve A u = f by conjugate gradients preconditioned with diag(A).

    Stops when ||f - A u||_2 <= tol ||f||_2, with the residual recomputed
    from u every 50 iterations (so the recursion's drift cannot fake
    convergence).  Returns (u, iterations, relative residual)."""
    f = np.asarray(f, dtype=np.float64)
    dinv = 1.0 / A.diagonal()
    u = np.zeros_like(f)
    r = f.copy()
    fn = np.linalg.norm(f)
    if fn == 0.0:
        return u, 0, 0.0
    z = dinv * r
    p = z.copy()
    rz = r @ z
    for it in range(1, max_iter + 1):
        Ap = A @ p
        alpha = rz / (p @ Ap)
        u += alpha * p
        if it % 50 == 0:
            r = f - A @ u
        else:
            r -= alpha * Ap
        rel = np.linalg.norm(r) / fn
        if rel <= tol:
            r = f - A @ u
            rel = np.linalg.norm(r) / fn
            if rel <= tol:
                return u, it, float(rel)
        z = dinv * r
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return u, max_iter, float(np.linalg.norm(f - A @ u) / fn)
