"""Pins for the oracle's column-pivoted QR and interpolative decomposition (§2.3)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import cpqr as cpqr_mod
from oracle.cpqr import cpqr, interpolative_decomposition


@pytest.mark.parametrize("shape,seed", [((30, 12), 0), ((100, 9), 1), ((12, 30), 2), ((64, 64), 3)])
def test_pivots_match_lapack(shape, seed):
    # LAPACK dgeqp3 (scipy.linalg.qr pivoting=True) is an independent CPQR
    M = np.random.default_rng(seed).standard_normal(shape)
    k, perm, R = cpqr(M, 0.0)
    Rl, Pl = sla.qr(M, mode="r", pivoting=True)
    kk = min(shape)
    assert k == kk
    assert np.array_equal(perm[:kk], Pl[:kk])
    assert np.allclose(np.abs(np.diag(R)), np.abs(np.diag(Rl))[:kk], rtol=1e-12)
    # R reproduces the permuted matrix: M[:, perm] = Q R  =>  R^T R = M_p^T M_p
    Mp = M[:, perm]
    assert np.allclose(R.T @ R, Mp.T @ Mp, rtol=0, atol=1e-10 * np.abs(Mp.T @ Mp).max())


def _decaying(m, n, decay, seed):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, min(m, n))))
    V, _ = np.linalg.qr(rng.standard_normal((n, min(m, n))))
    s = decay ** np.arange(min(m, n))
    return (U * s) @ V.T


@pytest.mark.parametrize("eps", [1e-2, 1e-4, 1e-6, 1e-9])
def test_id_error_bound(eps):
    # at termination every remaining column of the trailing block has norm
    # <= eps |R_11| <= eps ||M||_2, so ||M_red - M_skel T||_2 <= sqrt(n - k) eps ||M||_2
    M = _decaying(80, 40, 0.6, 5)
    k, skel, red, T = interpolative_decomposition(M, eps)
    err = np.linalg.norm(M[:, red] - M[:, skel] @ T, 2)
    assert err <= np.sqrt(max(red.size, 1)) * eps * np.linalg.norm(M, 2) * (1 + 1e-10)
    # and the rank is no smaller than the number of singular values above eps*sigma_1/sqrt(n)
    sv = np.linalg.svd(M, compute_uv=False)
    assert k >= np.sum(sv > eps * sv[0] * np.sqrt(M.shape[1]))
    assert k <= np.sum(sv > eps * sv[0] / np.sqrt(M.shape[1]) / 10)


def test_exact_low_rank():
    rng = np.random.default_rng(9)
    M = rng.standard_normal((50, 5)) @ rng.standard_normal((5, 16))
    k, skel, red, T = interpolative_decomposition(M, 1e-10)
    assert k == 5
    assert np.allclose(M[:, red], M[:, skel] @ T, atol=1e-11 * np.abs(M).max())


def test_zero_and_empty():
    k, skel, red, T = interpolative_decomposition(np.zeros((7, 4)), 1e-6)
    assert k == 0 and red.size == 4 and T.shape == (0, 4)
    k, skel, red, T = interpolative_decomposition(np.zeros((0, 4)), 1e-6)
    assert k == 0 and red.size == 4


def test_tie_breaks_to_lowest_index():
    # identical columns 0 and 1; column 2 is pivoted first and swapped into
    # position 0, so the current order is (2, 1, 0) and the tie goes to column 1
    M = np.array([[1.0, 1.0, 0.0], [0.0, 0.0, 2.0]])
    k, skel, red, T = interpolative_decomposition(M, 1e-12)
    assert list(skel) == [2, 1] and list(red) == [0]
    assert np.allclose(T, [[0.0], [1.0]])


def test_trace_records_the_pivot_norms_and_their_runner_up():
    # the trace's chosen norms are LAPACK's |R_ii| (dgeqp3); the runner-up is
    # the second largest column norm of the matrix with the chosen pivots'
    # directions projected out, computed here by brute force
    rng = np.random.default_rng(71)
    M = rng.standard_normal((40, 12)) @ np.diag(10.0 ** -np.arange(12))
    eps = 1e-7
    trace = []
    k, perm, R = cpqr(M, eps, trace)
    _, Rl, pl = sla.qr(M, pivoting=True, mode="economic")
    assert np.allclose([t[0] for t in trace[:k]], np.abs(np.diag(Rl))[:k], rtol=1e-10)
    for i in range(k):
        Q, _ = np.linalg.qr(M[:, perm[:i]]) if i else (np.zeros((40, 0)), None)
        P = M - Q @ (Q.T @ M)
        rest = [c for c in range(12) if c not in perm[:i]]
        nrm = np.sort(np.linalg.norm(P[:, rest], axis=0))[::-1]
        assert np.isclose(trace[i][0], nrm[0], rtol=1e-9)
        assert np.isclose(trace[i][1], nrm[1] if nrm.size > 1 else 0.0, rtol=1e-8, atol=1e-300)
        assert trace[i][2] == eps * trace[0][0]
    # the stop: the step after the last pivot saw a norm at or below eps |R_11|
    assert len(trace) == k + 1 and trace[k][0] <= trace[k][2]
    m = cpqr_mod.decision_margin(trace)
    assert 0.0 < m < 1.0


def test_decision_margin_is_zero_on_a_tie():
    # two columns of equal norm: the first pivot is a tie
    M = np.array([[3.0, 0.0, 1.0], [0.0, 3.0, 0.0], [0.0, 0.0, 0.5]])
    trace = []
    cpqr(M, 1e-12, trace)
    assert cpqr_mod.decision_margin(trace) == 0.0
