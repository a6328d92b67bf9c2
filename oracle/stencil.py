"""Seven-point finite-difference operator (oracle; test infrastructure only).

Follows the seven-point stencil equation of §2.4: at grid point j,

    (1/h^2) * sum_{d, +-} a_{j +- e_d/2} (u_j - u_{j +- e_d}) + b_j u_j = f_j .

Readings (the paper is periodic with h = 1/n and never defines the half-point
coefficients):
  * zero Dirichlet boundary on the n^3 interior grid of the unit cube,
    h = 1/(n+1); a neighbour outside the grid contributes its coupling to the
    diagonal only (u = 0 there);
  * a_{j +- e/2} is the harmonic mean 2 a_j a_k / (a_j + a_k) of the two grid
    values; towards the boundary it is a_j.

Index of grid point (j1, j2, j3) is j1 + n*j2 + n*n*j3.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def half_point_coefficients(a: np.ndarray, n: int):
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
        # last plane along the axis touches the boundary: use a_j
        idx_last = [slice(None)] * 3
        idx_last[axis] = n - 1
        harm[tuple(idx_last)] = a3[tuple(idx_last)]
        cp[d] = harm
        # a_{j - e/2} = a_{(j - e) + e/2}, and a_j on the first plane
        harm_m = np.roll(harm, 1, axis=axis)
        idx_first = [slice(None)] * 3
        idx_first[axis] = 0
        harm_m[tuple(idx_first)] = a3[tuple(idx_first)]
        cm[d] = harm_m
    return cm.reshape(3, -1), cp.reshape(3, -1)


def assemble(a: np.ndarray, b, n: int) -> sp.csr_matrix:
    """Sparse FP64 matrix A of the Dirichlet seven-point operator."""
    N = n * n * n
    h = 1.0 / (n + 1)
    inv_h2 = 1.0 / (h * h)
    bvec = np.broadcast_to(np.asarray(b, dtype=np.float64), (N,))
    cm, cp = half_point_coefficients(a, n)
    diag = inv_h2 * (cm.sum(axis=0) + cp.sum(axis=0)) + bvec
    rows = [np.arange(N)]
    cols = [np.arange(N)]
    vals = [diag]
    idx = np.arange(N)
    jc = [idx % n, (idx // n) % n, idx // (n * n)]
    stride = [1, n, n * n]
    for d in range(3):
        has_plus = jc[d] < n - 1
        src = idx[has_plus]
        dst = src + stride[d]
        w = -inv_h2 * cp[d][has_plus]
        rows += [src, dst]
        cols += [dst, src]
        vals += [w, w]
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, N)).tocsr()
    A.sum_duplicates()
    return A

