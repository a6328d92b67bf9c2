"""Hierarchical geometry of §2.1 (oracle; test infrastructure only).

At level l the cell side is s = m 2^l and the grid splits into c = n/s cells per
dimension.  In the paper (periodic) a cell owns its first frame as faces.  With
a zero Dirichlet boundary the first frame of the lowest cells touches the
boundary and separates nothing, so the reading used here is:

  coordinate j_d is a *separator* at level l  iff  j_d % s == 0 and j_d != 0.

A DOF with 0 / 1 / 2 / 3 separator coordinates is a cell interior / face /
edge / vertex point.  Faces exclude their edges and edges exclude vertices,
following the 3D HIF the paper builds on (cell structure figure of §2.1
distinguishes edge points).

Each coordinate is mapped to a *slab code*: separator plane j_d = k s -> 2k,
cell slab c (points strictly between planes) -> 2c + 1.  A group (cell
interior, face, edge, vertex) is the set of DOFs with equal code triples; the
number of even codes is the group's kind.  The closure of cell (2c+1, ...) is
every code triple with each code in {2c, 2c+1, 2c+2}.

Periodic grid (periodic=True, the paper's own setting): every multiple of s,
j_d = 0 included, is a separator, so each cell owns its first frame as in
§2.1, and codes are taken modulo 2c: the upper plane of the last cell is
plane 0.  The functions below take `ncode` = 2c (codes modulo ncode) for the
periodic grid and ncode = 0 for the Dirichlet one.
"""
from __future__ import annotations

import itertools

import numpy as np

KIND_CELL, KIND_FACE, KIND_EDGE, KIND_VERTEX = 0, 1, 2, 3


def num_levels(n: int, m: int) -> int:
    """L with n = m 2^L (§2.1); raises ValueError otherwise."""
    if n <= 0 or m <= 0 or n % m:
        raise ValueError(f"n={n} is not a multiple of m={m}")
    q = n // m
    L = q.bit_length() - 1
    if (1 << L) != q:
        raise ValueError(f"n/m = {q} is not a power of two")
    return L


def slab_codes(idx: np.ndarray, n: int, s: int, periodic: bool = False) -> np.ndarray:
    """Slab code triple (shape (len(idx), 3)) of each global DOF index at cell side s."""
    idx = np.asarray(idx, dtype=np.int64)
    out = np.empty((idx.size, 3), dtype=np.int64)
    for d, jd in enumerate((idx % n, (idx // n) % n, idx // (n * n))):
        sep = (jd % s == 0) if periodic else (jd % s == 0) & (jd != 0)
        out[:, d] = np.where(sep, 2 * (jd // s), 2 * (jd // s) + 1)
    return out


def group_active(active_idx: np.ndarray, n: int, s: int, periodic: bool = False) -> dict:
    """Map code triple -> sorted global indices of the active DOFs in that group."""
    active_idx = np.sort(np.asarray(active_idx, dtype=np.int64))
    codes = slab_codes(active_idx, n, s, periodic)
    if active_idx.size == 0:
        return {}
    key = (codes[:, 0] * (2 * n + 2) + codes[:, 1]) * (2 * n + 2) + codes[:, 2]
    order = np.argsort(key, kind="stable")
    key_sorted = key[order]
    starts = np.flatnonzero(np.r_[True, key_sorted[1:] != key_sorted[:-1]])
    ends = np.r_[starts[1:], key_sorted.size]
    groups = {}
    for a, b in zip(starts, ends):
        members = active_idx[order[a:b]]
        c = tuple(int(x) for x in codes[order[a]])
        groups[c] = np.sort(members)
    return groups


def kind(code) -> int:
    return sum(1 for x in code if x % 2 == 0)


def _wrap(c: int, ncode: int) -> int:
    return c % ncode if ncode else c


def cell_closure(code, ncode: int = 0) -> list:
    """All code triples in the closure of the cell with (all odd) code triple."""
    assert kind(code) == KIND_CELL
    return [tuple(t) for t in itertools.product(*[(c - 1, c, _wrap(c + 1, ncode)) for c in code])]


def adjacent_cells(code, ncode: int = 0) -> list:
    """Cells whose closure contains the group with this code triple."""
    choices = [(c,) if c % 2 else (_wrap(c - 1, ncode), c + 1) for c in code]
    return [tuple(t) for t in itertools.product(*choices)]


def count_groups(n: int, s: int, periodic: bool = False) -> dict:
    """Number of groups of each kind at cell side s when every DOF is active."""
    g = group_active(np.arange(n ** 3), n, s, periodic)
    out = {KIND_CELL: 0, KIND_FACE: 0, KIND_EDGE: 0, KIND_VERTEX: 0}
    for c in g:
        out[kind(c)] += 1
    return out
