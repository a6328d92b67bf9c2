"""Seven-point finite-difference operator (oracle; test infrastructure only).

Follows the seven-point stencil equation of §2.4: at grid point j,

    (1/h^2) * sum_{d, +-} a_{j +- e_d/2} (u_j - u_{j +- e_d}) + b_j u_j = f_j .

Readings (the paper is periodic with h = 1/n and never defines the half-point
coefficients):
  * default: zero Dirichlet boundary on the n^3 interior grid of the unit
    cube, h = 1/(n+1); a neighbour outside the grid contributes its coupling
    to the diagonal only (u = 0 there);
  * periodic=True: the paper's own setting, grid points j/n of the unit
    torus, h = 1/n; the neighbour of the last plane is the first plane (the
    operator is singular for b = 0, so b > 0 is needed);
  * a_{j +- e/2} is the harmonic mean 2 a_j a_k / (a_j + a_k) of the two grid
    values; towards a Dirichlet boundary it is a_j.

Index of grid point (j1, j2, j3) is j1 + n*j2 + n*n*j3.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def half_point_coefficients(a: np.ndarray, n: int, periodic: bool = False):
    """Return (cm, cp), each shape (3, n^3): a_{j - e_d/2} and a_{j + e_d/2}."""
    a3 = np.asarray(a, dtype=np.float64).reshape(n, n, n)  # [j3, j2, j1]
    cm = np.empty((3, n, n, n))
    cp = np.empty((3, n, n, n))
    for d in range(3):
        axis = 2 - d  # d = 0 -> j1 -> last numpy axis
        a_lo = a3
        # neighbour in +e_d direction
        a_nb = np.roll(a3, -1, axis=axis)
        harm = 2.0 * a_lo * a_nb / (a_lo + a_nb)
        if not periodic:
            # last plane along the axis touches the boundary: use a_j
            idx_last = [slice(None)] * 3
            idx_last[axis] = n - 1
            harm[tuple(idx_last)] = a3[tuple(idx_last)]
        cp[d] = harm
        # a_{j - e/2} = a_{(j - e) + e/2} (wrapping around when periodic), and
        # a_j on the first plane of a Dirichlet grid
        harm_m = np.roll(harm, 1, axis=axis)
        if not periodic:
            idx_first = [slice(None)] * 3
            idx_first[axis] = 0
            harm_m[tuple(idx_first)] = a3[tuple(idx_first)]
        cm[d] = harm_m
    return cm.reshape(3, -1), cp.reshape(3, -1)


def assemble(a: np.ndarray, b, n: int, periodic: bool = False) -> sp.csr_matrix:
    """Sparse FP64 matrix A of the seven-point operator (Dirichlet or periodic)."""
    N = n * n * n
    h = 1.0 / n if periodic else 1.0 / (n + 1)
    inv_h2 = 1.0 / (h * h)
    bvec = np.broadcast_to(np.asarray(b, dtype=np.float64), (N,))
    cm, cp = half_point_coefficients(a, n, periodic)
    diag = inv_h2 * (cm.sum(axis=0) + cp.sum(axis=0)) + bvec
    rows = [np.arange(N)]
    cols = [np.arange(N)]
    vals = [diag]
    idx = np.arange(N)
    jc = [idx % n, (idx // n) % n, idx // (n * n)]
    stride = [1, n, n * n]
    for d in range(3):
        has_plus = np.ones(N, dtype=bool) if periodic else jc[d] < n - 1
        src = idx[has_plus]
        # the +e_d neighbour, wrapping from the last plane to the first
        dst = src + np.where(jc[d][has_plus] < n - 1, stride[d], -(n - 1) * stride[d])
        w = -inv_h2 * cp[d][has_plus]
        rows += [src, dst]
        cols += [dst, src]
        vals += [w, w]
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, N)).tocsr()
    A.sum_duplicates()
    return A

