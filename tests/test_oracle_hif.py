"""Pins for the oracle's HIF factorization and application (§2.2-§2.4).

Independent references used here:
  * dense Cholesky solves of the assembled operator (numpy / LAPACK);
  * closed-form Dirichlet eigenpairs of the constant-coefficient operator;
  * the factorization's own definition: with W the product of the sparse
    factors S_I, Q_F S_F~ (built as dense matrices from the stored blocks) and
    the root factor, W^T A W = D = I (exactly at eps = 0, to O(eps) else), and
    F^{-1} = W W^T, which checks the sweep code of hif_apply separately.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import hif, krylov, stencil


def _problem(n, seed, lo=-1.0, hi=1.0, b=0.0):
    rng = np.random.default_rng(seed)
    a = 10.0 ** rng.uniform(lo, hi, n ** 3)
    return stencil.assemble(a, b, n)


def _dense_W(fac):
    """W = W^0 ... W^{L-1} W^L as a dense matrix, built from the records.

    S_I is the identity except rows I, which hold [L^{-T}, -L^{-T} X] on the
    columns (I, N).  For a face or edge the factor is Q_F S_F~ with Q_F the
    identity plus -T in rows F^, columns F~, and S_F~ like S_I on (F~, F^).
    Right-multiplying W by such a factor only rewrites the columns it touches.
    """
    N = fac.N
    W = np.eye(N)
    for r in fac.records:
        if isinstance(r, hif.CellRecord):
            Li = sla.solve_triangular(r.L, np.eye(r.I.size), lower=True).T   # L^{-T}
            WI = W[:, r.I].copy()
            W[:, r.I] = WI @ Li
            W[:, r.N] += WI @ (-Li @ r.X)
        else:
            W[:, r.Fc] -= W[:, r.Fh] @ r.T                                   # W Q_F
            Li = sla.solve_triangular(r.L, np.eye(r.Fc.size), lower=True).T
            Wc = W[:, r.Fc].copy()
            W[:, r.Fc] = Wc @ Li                                              # (W Q_F) S_F~
            W[:, r.Fh] += Wc @ (-Li @ r.X)
    S = fac.root.S
    W[:, S] = W[:, S] @ sla.solve_triangular(fac.root.L, np.eye(S.size), lower=True).T
    return W


@pytest.mark.parametrize("n,b", [(8, 0.0), (16, 0.3)])
def test_exact_mode_matches_dense_solve(n, b):
    A = _problem(n, 11, b=b)
    fac = hif.hif_factor(A, n, 4, 0.0)
    f = np.random.default_rng(12).standard_normal((3, n ** 3))
    u = hif.hif_apply(fac, f)
    c = sla.cho_factor(A.toarray())
    ref = sla.cho_solve(c, f.T).T
    assert np.linalg.norm(u - ref) <= 1e-10 * np.linalg.norm(ref)


def test_exact_mode_eigenvectors():
    n = 16
    A = stencil.assemble(np.ones(n ** 3), 0.0, n)
    fac = hif.hif_factor(A, n, 4, 0.0)
    h = 1.0 / (n + 1)
    idx = np.arange(n ** 3)
    coords = [idx % n, (idx // n) % n, idx // (n * n)]
    for p in [(1, 1, 1), (3, 7, 2), (16, 16, 16)]:
        v = np.ones(n ** 3)
        lam = 0.0
        for d in range(3):
            v = v * np.sin(p[d] * np.pi * (coords[d] + 1) * h)
            lam += 4.0 / h ** 2 * np.sin(p[d] * np.pi * h / 2) ** 2
        assert np.allclose(hif.hif_apply(fac, v), v / lam, rtol=0, atol=1e-10 * np.abs(v).max() / lam)


@pytest.mark.parametrize("eps", [0.0, 1e-6])
def test_congruence_identity(eps):
    # W^T A W = I: exact at eps = 0; at eps > 0 the dropped blocks are O(eps)
    n = 8 if eps == 0 else 16
    A = _problem(n, 21)
    fac = hif.hif_factor(A, n, 4, eps)
    W = _dense_W(fac)
    E = W.T @ (A @ W) - np.eye(n ** 3)
    err = np.abs(E).max()
    if eps == 0:
        assert err < 1e-10
    else:
        assert err < 1e3 * eps
    # F^{-1} = W W^T: the apply sweeps agree with the dense product
    f = np.random.default_rng(22).standard_normal(n ** 3)
    assert np.allclose(hif.hif_apply(fac, f), W @ (W.T @ f), rtol=0,
                       atol=1e-11 * np.abs(W @ (W.T @ f)).max())


def test_skeletonization_happens_and_is_symmetric():
    n = 16
    A = _problem(n, 31)
    fac = hif.hif_factor(A, n, 4, 1e-3)
    assert any(isinstance(r, hif.SkelRecord) for r in fac.records)
    assert fac.root_size < n ** 3 - (n - 1) ** 3
    rng = np.random.default_rng(32)
    x, y = rng.standard_normal((2, n ** 3))
    fx, fy = hif.hif_apply(fac, x), hif.hif_apply(fac, y)
    assert abs(x @ fy - y @ fx) <= 1e-13 * np.linalg.norm(x) * np.linalg.norm(fy)
    assert x @ fx > 0 and y @ fy > 0


def test_error_scales_with_eps():
    # e_s and max|1 - lambda(F^{-1}A)| shrink with eps and stay near eps for a = 1
    n = 16
    A = stencil.assemble(np.ones(n ** 3), 0.0, n)
    rng = np.random.default_rng(41)
    x = rng.standard_normal(n ** 3)
    v0 = rng.standard_normal(n ** 3)
    es, pn = [], []
    for eps in (1e-2, 1e-4, 1e-6):
        fac = hif.hif_factor(A, n, 4, eps)
        es.append(krylov.solve_error(A, fac, x))
        pn.append(krylov.power_norm(A, fac, v0, iters=30))
        assert 1e-3 * eps < es[-1] < 10 * eps
        assert pn[-1] < 30 * eps
    assert es[0] > es[1] > es[2]
    assert pn[0] > pn[1] > pn[2]


def test_pcg_converges_to_dense_solution():
    n = 16
    A = _problem(n, 51, b=0.1)
    fac = hif.hif_factor(A, n, 4, 1e-3)
    f = np.random.default_rng(52).standard_normal(n ** 3)
    u, it, hist = krylov.pcg(A, fac, f, tol=1e-10)
    assert hist[-1] <= 1e-10 and it <= 15
    ref = sla.cho_solve(sla.cho_factor(A.toarray()), f)
    assert np.linalg.norm(u - ref) <= 1e-8 * np.linalg.norm(ref)


def test_locality_assertion_is_live():
    # the factorization asserts that each front couples only inside its closure;
    # a coupling planted across two far cells must trip it
    n = 16
    A = _problem(n, 61).tolil()
    A[0, n ** 3 - 1] = -1e-3
    A[n ** 3 - 1, 0] = -1e-3
    with pytest.raises(AssertionError):
        hif.hif_factor(A.tocsr(), n, 4, 0.0)


# ---- planted mistakes: each one must be caught by a pin above -----------------

def test_planted_transposed_interpolation_is_caught(monkeypatch):
    import oracle.hif as H
    real = H.interpolative_decomposition

    def bad(M, eps, trace=None):
        k, s, r, T = real(M, eps, trace)
        if T.size and T.shape[0] == T.shape[1]:
            T = T.T
        elif T.size:
            T = -T
        return k, s, r, T

    monkeypatch.setattr(H, "interpolative_decomposition", bad)
    n = 16
    A = _problem(n, 21)
    fac = hif.hif_factor(A, n, 4, 1e-6)
    W = _dense_W(fac)
    assert np.abs(W.T @ (A @ W) - np.eye(n ** 3)).max() > 1e3 * 1e-6


def test_planted_dropped_schur_term_is_caught(monkeypatch):
    import oracle.hif as H
    real = H.sla.solve_triangular
    calls = {"n": 0}

    def bad(Lm, B, **kw):
        out = real(Lm, B, **kw)
        calls["n"] += 1
        return 0.5 * out if calls["n"] == 3 else out   # one wrong X block

    monkeypatch.setattr(H.sla, "solve_triangular", bad)
    n = 8
    A = _problem(n, 11)
    fac = hif.hif_factor(A, n, 4, 0.0)
    monkeypatch.setattr(H.sla, "solve_triangular", real)
    f = np.random.default_rng(12).standard_normal(n ** 3)
    ref = sla.cho_solve(sla.cho_factor(A.toarray()), f)
    assert np.linalg.norm(hif.hif_apply(fac, f) - ref) > 1e-6 * np.linalg.norm(ref)


# ---- periodic grid -------------------------------------------------------------

@pytest.mark.parametrize("n,m,b", [(8, 4, 0.3), (12, 3, 1.0)])
def test_periodic_exact_mode_matches_dense_solve(n, m, b):
    rng = np.random.default_rng(21)
    A = stencil.assemble(10.0 ** rng.uniform(-1, 1, n ** 3), b, n, periodic=True)
    fac = hif.hif_factor(A, n, m, 0.0, periodic=True)
    # eps = 0: the root keeps the separator planes of the last level, n^3 - (n - 2)^3
    assert fac.root.S.size == n ** 3 - (n - 2) ** 3
    f = rng.standard_normal((2, n ** 3))
    u = hif.hif_apply(fac, f)
    ref = sla.cho_solve(sla.cho_factor(A.toarray()), f.T).T
    assert np.linalg.norm(u - ref) <= 1e-10 * np.linalg.norm(ref)


def test_periodic_error_scales_with_eps():
    # a well-conditioned periodic problem (b = 20 keeps the smallest
    # eigenvalue well above the compression error): e_s falls with eps
    n = 16
    rng = np.random.default_rng(22)
    A = stencil.assemble(10.0 ** rng.uniform(-1, 1, n ** 3), 20.0, n, periodic=True)
    x = rng.standard_normal(n ** 3)
    es = []
    for eps in (1e-2, 1e-4):
        fac = hif.hif_factor(A, n, 4, eps, periodic=True)
        es.append(np.linalg.norm(x - hif.hif_apply(fac, A @ x)) / np.linalg.norm(x))
    assert es[1] < es[0] < 0.5 and es[1] < 1e-2


def _golden(name):
    import os
    out = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                out[k] = float(v)
    return out


def test_periodic_example1_matches_the_papers_table():
    # the paper's Example 1 at 32^3 (periodic, a = 1, b = 0.1 against the
    # unscaled stencil, eps = 1e-3): the oracle keeps exactly the printed
    # number of top-level points and its e_s lies in the printed range
    g = _golden("example1_periodic_32.txt")
    n, m = int(g["n"]), int(g["m"])
    A = stencil.assemble(np.ones(n ** 3), g["b_over_stencil"] * n * n, n, periodic=True)
    fac = hif.hif_factor(A, n, m, g["eps"], check=False, periodic=True)
    assert fac.root.S.size == int(g["root_size"])
    x = np.random.default_rng(2).standard_normal(n ** 3)
    es = np.linalg.norm(x - hif.hif_apply(fac, A @ x)) / np.linalg.norm(x)
    assert g["es_min"] <= es <= g["es_max"], es


def test_recorded_active_sets_follow_the_records():
    # record=True keeps the active set after every level and every ID's
    # decision; both must agree with the stored factors: the DOFs active after
    # level l are those active before it minus the level's eliminated cell
    # interiors and the redundant DOFs of its faces and edges
    n, eps = 16, 1e-4
    A = _problem(n, 91)
    fac = hif.hif_factor(A, n, 4, eps, record=True)
    before = np.arange(n ** 3)
    for lev, act in enumerate(fac.active):
        gone = [r.I for r in fac.records if isinstance(r, hif.CellRecord) and r.level == lev]
        gone += [np.setdiff1d(F, skel) for (l, _, F, skel, _) in fac.ids if l == lev]
        expect = np.setdiff1d(before, np.concatenate(gone))
        assert np.array_equal(act, expect)
        assert act.size == fac.ranks[lev][1]
        before = act
    assert np.array_equal(fac.active[-1], fac.root.S)
    for (l, kind, F, skel, marg) in fac.ids:
        assert np.all(np.isin(skel, F)) and marg >= 0.0
    # recording changes nothing in the factorization
    plain = hif.hif_factor(A, n, 4, eps)
    x = np.random.default_rng(92).standard_normal(n ** 3)
    assert np.array_equal(hif.hif_apply(plain, x), hif.hif_apply(fac, x))


@pytest.mark.parametrize("n,lo,hi", [(8, -2.0, 2.0), (12, -1.0, 1.0)])
def test_jacobi_cg_matches_dense_solve(n, lo, hi):
    A = _problem(n, 93 + n, lo=lo, hi=hi, b=0.1)
    f = np.random.default_rng(94).standard_normal(n ** 3)
    u, its, rel = krylov.cg_jacobi(A, f, tol=1e-14)
    ref = sla.cho_solve(sla.cho_factor(A.toarray()), f)
    assert rel <= 1e-14 and np.linalg.norm(f - A @ u) <= 1e-14 * np.linalg.norm(f)
    assert np.linalg.norm(u - ref) <= 1e-11 * np.linalg.norm(ref)


def test_jacobi_cg_solves_an_eigenvector_exactly():
    # constant a: v_j = prod_d sin(p_d pi (j_d + 1) h) is an eigenvector with
    # lambda = (4/h^2) sum_d sin^2(p_d pi h / 2), so A u = v gives u = v / lambda
    n, p = 10, (1, 2, 3)
    h = 1.0 / (n + 1)
    A = stencil.assemble(np.ones(n ** 3), 0.0, n)
    j = np.arange(n)
    v = np.einsum("k,j,i->kji", *[np.sin(q * np.pi * (j + 1) * h) for q in p[::-1]]).reshape(-1)
    lam = 4.0 / h ** 2 * sum(np.sin(q * np.pi * h / 2) ** 2 for q in p)
    u, its, rel = krylov.cg_jacobi(A, v, tol=1e-14)
    assert np.linalg.norm(u - v / lam) <= 1e-12 * np.linalg.norm(v / lam)
