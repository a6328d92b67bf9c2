"""Sequential HIF factorization and application of F^{-1} (oracle; test infrastructure only).

Follows §2.4 ("Sequential HIF") in the paper's order:

  for l = 0 .. L-1:
    * sparse elimination (§2.2) of every cell interior I:  A_II = L L^T,
      X = L^{-1} A_IN, and the Schur update A_NN -= X^T X;
    * skeletonization (§2.3) of every face F with the ID of A_RF, then the same
      for every edge (faces exclude edges, see geometry.py);
    * Sigma^{l+1} = Sigma^l minus the eliminated interiors and redundant DOFs;
  level L: Cholesky of A^L restricted to Sigma^L;

and then F^{-1} = W^0 ... W^{L-1} W^L D^{-1} W^{L T} ... W^{0 T}.

Readings (the paper is silent or ambiguous on these):
  * LDL^T is taken as Cholesky (D = I): A is SPD for b >= 0 with the Dirichlet
    boundary, and so are all Schur complements.  On the periodic grid A is
    SPD only for b > 0, its smallest eigenvalue is about b, and a compression
    error above that can leave an indefinite Schur complement (the paper's
    LDL^T with GMRES covers that case; Cholesky then stops at the root);
  * faces of a level are skeletonized independently, each from the matrix as
    it stands after that level's cell eliminations (the distributed algorithm
    of §3.2 does them concurrently); edges likewise, after all faces;
  * the per-front congruence is Q_F then S_F~ (eq. of §2.3 that factorizes
    S^T Q^T A Q S); the product written over all faces in §2.4 lists the
    factors in the other order, which is read as a typo;
  * eps = 0 skips the ID: every face DOF is a skeleton and HIF reduces to
    exact nested-dissection multifrontal elimination.

Storage: A^l is a scipy CSR matrix over the global indices.  Eliminated DOFs
get zero rows and columns.  Dense blocks are pulled out with fancy indexing.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import geometry as geo
from .cpqr import interpolative_decomposition


@dataclass
class CellRecord:          # S_I of §2.2 with D_I = I
    level: int
    I: np.ndarray          # eliminated interior DOFs
    N: np.ndarray          # surrounding active DOFs (rest of the cell closure)
    L: np.ndarray          # A_II = L L^T
    X: np.ndarray          # L^{-1} A_IN   (|I| x |N|)


@dataclass
class SkelRecord:          # Q_F and S_F~ of §2.3
    level: int
    kind: int              # geo.KIND_FACE or geo.KIND_EDGE
    Fc: np.ndarray         # redundant DOFs F~ (eliminated)
    Fh: np.ndarray         # skeleton DOFs F^ (stay active)
    T: np.ndarray          # interpolation matrix, |F^| x |F~|
    L: np.ndarray          # B_{F~F~} = L L^T
    X: np.ndarray          # L^{-1} B_{F^F~}^T   (|F~| x |F^|)


@dataclass
class RootRecord:          # W^L of §2.4, level L
    S: np.ndarray
    L: np.ndarray


@dataclass
class Factor:
    n: int
    m: int
    eps: float
    records: list = field(default_factory=list)
    root: RootRecord | None = None
    ranks: list = field(default_factory=list)   # per level: (|Sigma^l| before, after)
    flops: float = 0.0                          # algorithmic flop count (Cholesky k^3/3, TRSM, GEMM 2mnk)
    # test instrumentation, filled when hif_factor(..., record=True):
    # active[l] = sorted DOFs of Sigma^{l+1} (active after level l); ids =
    # every ID of the factorization as (level, kind, F, skeleton DOFs,
    # decision margin of its CPQR, see cpqr.decision_margin)
    active: list = field(default_factory=list)
    ids: list = field(default_factory=list)

    @property
    def N(self):
        return self.n ** 3

    @property
    def root_size(self):
        return 0 if self.root is None else int(self.root.S.size)

    def stored_entries(self) -> int:
        """Number of stored factor entries (triangles counted in full)."""
        tot = 0
        for r in self.records:
            tot += r.L.size + r.X.size
            if isinstance(r, SkelRecord):
                tot += r.T.size
        if self.root is not None:
            tot += self.root.L.size
        return tot


def _dense(A: sp.csr_matrix, rows, cols) -> np.ndarray:
    return A[rows][:, cols].toarray()


def _zero_rows_cols(A: sp.csr_matrix, idx: np.ndarray) -> sp.csr_matrix:
    keep = np.ones(A.shape[0])
    keep[idx] = 0.0
    D = sp.diags(keep)
    A = (D @ A @ D).tocsr()
    A.eliminate_zeros()
    return A


def _closure_dofs(groups: dict, cell_codes, exclude, ncode: int = 0) -> np.ndarray:
    """Active DOFs in the union of the closures of the given cells, minus `exclude`."""
    seen = set()
    parts = []
    for cc in cell_codes:
        for g in geo.cell_closure(cc, ncode):
            if g in groups and g not in seen and g != exclude:
                seen.add(g)
                parts.append(groups[g])
    if not parts:
        return np.zeros(0, dtype=np.int64)
    return np.sort(np.concatenate(parts))


def _check_local(A: sp.csr_matrix, rows: np.ndarray, allowed: np.ndarray):
    """Assert that rows couple only to `allowed` columns (locality of §2.4)."""
    sub = A[rows]
    cols = np.unique(sub.indices[sub.data != 0])
    extra = np.setdiff1d(cols, allowed, assume_unique=True)
    if extra.size:
        raise AssertionError(f"front couples to {extra.size} DOFs outside its closure")


def _eliminate_cells(A, groups, level, fac: Factor, check: bool, ncode: int = 0):
    rows, cols, vals = [], [], []
    eliminated = []
    for code, I in groups.items():
        if geo.kind(code) != geo.KIND_CELL:
            continue
        N = _closure_dofs(groups, [code], exclude=code, ncode=ncode)
        if check:
            _check_local(A, I, np.union1d(I, N))
        A_II = _dense(A, I, I)
        A_IN = _dense(A, I, N)
        Lc = sla.cholesky(A_II, lower=True)
        X = sla.solve_triangular(Lc, A_IN, lower=True)
        S = X.T @ X
        ni, nn = I.size, N.size
        fac.flops += ni ** 3 / 3.0 + ni * ni * nn + 2.0 * nn * nn * ni
        fac.records.append(CellRecord(level, I, N, Lc, X))
        r, c = np.meshgrid(N, N, indexing="ij")
        rows.append(r.ravel())
        cols.append(c.ravel())
        vals.append(-S.ravel())
        eliminated.append(I)
    if rows:
        upd = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                            shape=A.shape).tocsr()
        A = (A + upd).tocsr()
    if eliminated:
        A = _zero_rows_cols(A, np.concatenate(eliminated))
    return A, (np.concatenate(eliminated) if eliminated else np.zeros(0, np.int64))


def _skeletonize(A, groups, level, want_kind, eps, fac: Factor, check: bool, ncode: int = 0,
                 record: bool = False):
    """Skeletonize every group of `want_kind` independently (level-synchronous)."""
    from .cpqr import decision_margin
    rows, cols, vals = [], [], []
    redundant = []
    for code, F in groups.items():
        if geo.kind(code) != want_kind or F.size == 0:
            continue
        R = _closure_dofs(groups, geo.adjacent_cells(code, ncode), exclude=code, ncode=ncode)
        if check:
            _check_local(A, F, np.union1d(F, R))
        A_RF = _dense(A, R, F)
        trace = [] if record else None
        k, skel, red, T = interpolative_decomposition(A_RF, eps, trace)
        if record:
            fac.ids.append((level, want_kind, F, F[skel], decision_margin(trace)))
        fac.flops += 2.0 * R.size * F.size * F.size
        if red.size == 0:
            continue
        A_FF = _dense(A, F, F)
        A_hh = A_FF[np.ix_(skel, skel)]
        A_hc = A_FF[np.ix_(skel, red)]
        A_cc = A_FF[np.ix_(red, red)]
        # §2.3: B_{F~F~}, B_{F^F~}, then LDL^T (here Cholesky) of B_{F~F~}
        B_cc = A_cc - T.T @ A_hc - A_hc.T @ T + T.T @ A_hh @ T
        B_hc = A_hc - A_hh @ T
        Lf = sla.cholesky(B_cc, lower=True)
        X = sla.solve_triangular(Lf, B_hc.T, lower=True)
        # B_{F^F^} = A_{F^F^} - B_{F^F~} B_{F~F~}^{-1} B_{F^F~}^T = A_{F^F^} - X^T X
        XtX = X.T @ X
        nc, nh = red.size, skel.size
        fac.flops += nc ** 3 / 3.0 + nc * nc * nh + 2.0 * nh * nh * nc
        Fh, Fc = F[skel], F[red]
        fac.records.append(SkelRecord(level, want_kind, Fc, Fh, T, Lf, X))
        if nh:
            r, c = np.meshgrid(Fh, Fh, indexing="ij")
            rows.append(r.ravel())
            cols.append(c.ravel())
            vals.append(-XtX.ravel())
        redundant.append(Fc)
    if not redundant:
        return A, np.zeros(0, np.int64)
    if rows:
        upd = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                            shape=A.shape).tocsr()
        A = (A + upd).tocsr()
    red_all = np.concatenate(redundant)
    A = _zero_rows_cols(A, red_all)
    return A, red_all


def hif_factor(A0: sp.spmatrix, n: int, m: int, eps: float, check: bool = True,
               periodic: bool = False, record: bool = False) -> Factor:
    """Factor A ~= F per §2.4 and return the sparse factors W^0..W^L.

    periodic=True takes the periodic geometry (every multiple of the cell side
    is a separator and the cells wrap around, see geometry.py); A0 must then be
    the periodic operator.  record=True keeps the active set after every
    level and the decisions of every ID (Factor.active, Factor.ids)."""
    L = geo.num_levels(n, m)
    A = sp.csr_matrix(A0, dtype=np.float64, copy=True)
    fac = Factor(n=n, m=m, eps=float(eps))
    active = np.ones(n ** 3, dtype=bool)
    for level in range(L):
        s = m << level
        before = int(active.sum())
        ncode = 2 * (n // s) if periodic else 0
        groups = geo.group_active(np.flatnonzero(active), n, s, periodic)
        A, elim = _eliminate_cells(A, groups, level, fac, check, ncode)
        active[elim] = False
        if eps > 0.0:
            for want in (geo.KIND_FACE, geo.KIND_EDGE):
                groups = geo.group_active(np.flatnonzero(active), n, s, periodic)
                A, red = _skeletonize(A, groups, level, want, eps, fac, check, ncode, record)
                active[red] = False
        fac.ranks.append((before, int(active.sum())))
        if record:
            fac.active.append(np.flatnonzero(active))
    S = np.flatnonzero(active)
    A_SS = _dense(A, S, S)
    fac.root = RootRecord(S, sla.cholesky(A_SS, lower=True))
    fac.flops += S.size ** 3 / 3.0
    return fac


def _trsm(Lm, y, trans=False):
    return sla.solve_triangular(Lm, y, lower=True, trans="T" if trans else "N")


def hif_apply(fac: Factor, f: np.ndarray) -> np.ndarray:
    """u = F^{-1} f.  f has shape (N,) or (nrhs, N)."""
    f = np.asarray(f, dtype=np.float64)
    one = f.ndim == 1
    y = (f[None, :] if one else f).T.copy()       # N x nrhs
    # forward: W^{0T}, ..., W^{(L-1)T}
    for r in fac.records:
        if isinstance(r, CellRecord):
            yI = _trsm(r.L, y[r.I])
            y[r.I] = yI
            y[r.N] -= r.X.T @ yI
        else:
            y[r.Fc] -= r.T.T @ y[r.Fh]
            yc = _trsm(r.L, y[r.Fc])
            y[r.Fc] = yc
            y[r.Fh] -= r.X.T @ yc
    # level L: D^{-1} with W^L = L_Sigma^{-T} on Sigma^L (D = I on inactive DOFs)
    if fac.root is not None and fac.root.S.size:
        S = fac.root.S
        y[S] = _trsm(fac.root.L, _trsm(fac.root.L, y[S]), trans=True)
    # backward: W^{L-1}, ..., W^0
    for r in reversed(fac.records):
        if isinstance(r, CellRecord):
            y[r.I] = _trsm(r.L, y[r.I] - r.X @ y[r.N], trans=True)
        else:
            y[r.Fc] = _trsm(r.L, y[r.Fc] - r.X @ y[r.Fh], trans=True)
            y[r.Fh] -= r.T @ y[r.Fc]
    out = y.T
    return out[0].copy() if one else np.ascontiguousarray(out)
