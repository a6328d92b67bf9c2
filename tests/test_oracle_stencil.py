"""Pins for the oracle's seven-point operator (§2.4, seven-point stencil equation)."""
import os

import numpy as np
import pytest

from oracle import stencil

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _eig(n, p):
    # closed-form Dirichlet eigenpair of the 7-point Laplacian (a = 1, b = 0):
    # v_j = prod_d sin(p_d pi (j_d+1) h), lambda = (4/h^2) sum_d sin^2(p_d pi h/2)
    h = 1.0 / (n + 1)
    idx = np.arange(n ** 3)
    coords = [idx % n, (idx // n) % n, idx // (n * n)]
    v = np.ones(n ** 3)
    s = 0.0
    for d in range(3):
        v = v * np.sin(p[d] * np.pi * (coords[d] + 1) * h)
        s += np.sin(p[d] * np.pi * h / 2) ** 2
    return 4.0 * s / h ** 2, v


@pytest.mark.parametrize("n,p", [(5, (1, 1, 1)), (8, (1, 2, 3)), (8, (8, 1, 5)), (7, (4, 4, 4))])
def test_dirichlet_eigenpairs(n, p):
    A = stencil.assemble(np.ones(n ** 3), 0.0, n)
    lam, v = _eig(n, p)
    r = A @ v - lam * v
    assert np.linalg.norm(r) <= 1e-12 * lam * np.linalg.norm(v)


def test_constant_b_shifts_spectrum():
    n = 6
    A = stencil.assemble(np.ones(n ** 3), 0.25, n)
    lam, v = _eig(n, (2, 3, 1))
    assert np.allclose(A @ v, (lam + 0.25) * v, rtol=0, atol=1e-10 * lam)


def test_golden_hand_derived_entries():
    A = stencil.assemble(np.arange(1, 9, dtype=float), 0.5, 2).toarray()
    rows = [l.split() for l in open(os.path.join(GOLDEN, "stencil_n2.txt"))
            if l.strip() and not l.startswith("#")]
    for r, c, v in rows:
        assert A[int(r), int(c)] == pytest.approx(float(v), rel=1e-14, abs=1e-12)


def test_symmetric_and_row_sums():
    n = 6
    rng = np.random.default_rng(3)
    a = 10.0 ** rng.uniform(-2, 2, n ** 3)
    A = stencil.assemble(a, 0.0, n)
    assert abs(A - A.T).max() == 0.0
    # with a = 1, b = 0 a row sums to (#boundary neighbours)/h^2
    A1 = stencil.assemble(np.ones(n ** 3), 0.0, n)
    idx = np.arange(n ** 3)
    nb = sum(((c == 0).astype(int) + (c == n - 1).astype(int))
             for c in (idx % n, (idx // n) % n, idx // (n * n)))
    h = 1.0 / (n + 1)
    assert np.allclose(np.asarray(A1.sum(axis=1)).ravel(), nb / h ** 2, rtol=1e-13)


def test_positive_definite_small():
    n = 4
    rng = np.random.default_rng(4)
    a = 10.0 ** rng.uniform(-1, 1, n ** 3)
    A = stencil.assemble(a, 0.0, n).toarray()
    assert np.linalg.eigvalsh(A).min() > 0


# ---- periodic grid (the paper's own setting, h = 1/n) ---------------------------

def _periodic_eig(n, k):
    # Fourier eigenpair of the periodic 7-point Laplacian (a = 1):
    # v_j = prod_d cos(2 pi k_d j_d / n), lambda = (4/h^2) sum_d sin^2(pi k_d / n)
    h = 1.0 / n
    idx = np.arange(n ** 3)
    coords = [idx % n, (idx // n) % n, idx // (n * n)]
    v = np.ones(n ** 3)
    s = 0.0
    for d in range(3):
        v = v * np.cos(2.0 * np.pi * k[d] * coords[d] / n)
        s += np.sin(np.pi * k[d] / n) ** 2
    return 4.0 * s / h ** 2, v


@pytest.mark.parametrize("n,k", [(6, (1, 0, 2)), (8, (1, 2, 3)), (8, (4, 4, 1)), (5, (2, 1, 1))])
def test_periodic_fourier_eigenpairs(n, k):
    b = 0.3
    A = stencil.assemble(np.ones(n ** 3), b, n, periodic=True)
    lam, v = _periodic_eig(n, k)
    r = A @ v - (lam + b) * v
    assert np.linalg.norm(r) <= 1e-12 * (lam + b) * np.linalg.norm(v)


def test_periodic_rows_sum_to_b_and_wrap():
    # every coupling of the periodic operator has its mirror on the diagonal,
    # so A 1 = b for any positive a; the first and last planes are coupled
    n = 5
    rng = np.random.default_rng(3)
    a = 10.0 ** rng.uniform(-2, 2, n ** 3)
    bvec = rng.uniform(0.1, 1.0, n ** 3)
    A = stencil.assemble(a, bvec, n, periodic=True)
    assert np.allclose(A @ np.ones(n ** 3), bvec, rtol=0, atol=1e-9 * abs(A).max())
    assert abs(A - A.T).max() == 0.0
    j_first, j_last = 0, n - 1            # (j1, 0, 0) neighbours across the wrap
    harm = 2.0 * a[j_first] * a[j_last] / (a[j_first] + a[j_last])
    assert A[j_first, j_last] == pytest.approx(-harm * n * n, rel=1e-14)
