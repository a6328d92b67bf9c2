"""Interpolative decomposition by column-pivoted QR (oracle; test infrastructure only).

§2.3: the ID of A_RF writes (up to a permutation) A_RF = [A_{R,F~} A_{R,F^}]
~= [A_{R,F^} T_F, A_{R,F^}], with skeleton F^, redundant F~ and interpolation
matrix T_F.  The paper computes it with a pivoting QR (§3.3.2) to a relative
precision eps (Table 2).

Plain Householder QR with column pivoting, written from its definition: at
step i the remaining column of largest 2-norm (recomputed from scratch, no
downdating) is swapped to position i and a Householder reflector zeroes it
below the diagonal.  Readings:
  * rank k = number of steps with |R_ii| > eps |R_11| (the pivots of CPQR are
    non-increasing, so the loop stops at the first failure);
  * ties between equal column norms go to the lowest current column index;
  * A_RF = 0 (or no rows) gives k = 0: every DOF of F is redundant;
  * T_F = R11^{-1} R12.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def cpqr(M: np.ndarray, eps: float, trace: list | None = None):
    """Column-pivoted QR stopped at tolerance eps.

    Returns (k, perm, R) where perm is the column permutation (perm[:k] are the
    pivot columns) and R is the k x ncols upper-trapezoidal factor of the
    permuted matrix.

    With a list `trace`, each step appends (largest remaining column norm,
    second largest, eps |R_11|): how clearly the pivot and the stop were
    decided (test instrumentation; the arithmetic is the same either way).
    """
    W = np.array(M, dtype=np.float64, copy=True)
    m, n = W.shape
    perm = np.arange(n)
    kmax = min(m, n)
    k = kmax
    r11 = 0.0
    for i in range(kmax):
        norms = np.sqrt(np.sum(W[i:, i:] ** 2, axis=0))
        p = int(np.argmax(norms))  # first maximum = lowest current index
        if trace is not None:
            second = float(np.partition(norms, -2)[-2]) if norms.size > 1 else 0.0
            trace.append((float(norms[p]), second, eps * (norms[p] if i == 0 else r11)))
        if i == 0:
            r11 = norms[p]
            if r11 == 0.0:
                k = 0
                break
        if not norms[p] > eps * r11:
            k = i
            break
        if p:
            W[:, [i, i + p]] = W[:, [i + p, i]]
            perm[[i, i + p]] = perm[[i + p, i]]
        x = W[i:, i].copy()
        alpha = -np.copysign(np.linalg.norm(x), x[0])
        v = x
        v[0] -= alpha
        vnorm = np.linalg.norm(v)
        if vnorm > 0.0:
            v /= vnorm
            W[i:, i:] -= 2.0 * np.outer(v, v @ W[i:, i:])
        W[i + 1:, i] = 0.0
    return k, perm, np.triu(W[:k, :])


def decision_margin(trace: list) -> float:
    """Smallest relative gap of a traced CPQR: between the chosen and the next
    column norm at every pivot step, and between the last norms seen and the
    stopping threshold eps |R_11|.  Inputs perturbed by less than this
    (relative) make the same choices."""
    marg = np.inf
    for best, second, thr in trace:
        if best > 0.0:
            marg = min(marg, (best - second) / best)
        if thr > 0.0:
            marg = min(marg, abs(best - thr) / thr)
    return float(marg)


def interpolative_decomposition(M: np.ndarray, eps: float, trace: list | None = None):
    """ID of M (rows R, columns F) to relative precision eps.

    Returns (k, skel, redund, T): local column indices of the skeleton F^ and
    the redundant set F~ and T (k x |F~|) with M[:, redund] ~= M[:, skel] @ T.
    `trace` as for cpqr.
    """
    k, perm, R = cpqr(M, eps, trace)
    skel = perm[:k]
    redund = perm[k:]
    if k == 0:
        T = np.zeros((0, redund.size))
    else:
        T = sla.solve_triangular(R[:, :k], R[:, k:], lower=False)
    return k, skel, redund, T
