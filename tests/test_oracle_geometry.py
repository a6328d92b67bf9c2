"""Pins for the oracle's hierarchical geometry (§2.1) on the Dirichlet grid."""
import numpy as np
import pytest

from oracle import geometry as geo
from oracle import hif, stencil


@pytest.mark.parametrize("n,m", [(16, 4), (32, 4), (64, 4), (24, 3), (48, 3)])
def test_group_counts_closed_form(n, m):
    L = geo.num_levels(n, m)
    for level in range(L + 1):
        s = m << level
        c = n // s
        got = geo.count_groups(n, s)
        # c^3 cells, 3(c-1)c^2 faces, 3(c-1)^2 c edges, (c-1)^3 vertices
        assert got[geo.KIND_CELL] == c ** 3
        assert got[geo.KIND_FACE] == 3 * (c - 1) * c * c
        assert got[geo.KIND_EDGE] == 3 * (c - 1) ** 2 * c
        assert got[geo.KIND_VERTEX] == (c - 1) ** 3


def test_num_levels():
    assert geo.num_levels(16, 4) == 2
    assert geo.num_levels(128, 4) == 5
    assert geo.num_levels(96, 3) == 5
    with pytest.raises(ValueError):
        geo.num_levels(20, 4)
    with pytest.raises(ValueError):
        geo.num_levels(18, 4)


def test_face_sizes_level0():
    # level 0, m = 4: interior faces are 3x3, faces touching the low boundary 3x4 or 4x4
    g = geo.group_active(np.arange(16 ** 3), 16, 4)
    sizes = sorted({v.size for k, v in g.items() if geo.kind(k) == geo.KIND_FACE})
    assert sizes == [9, 12, 16]
    cells = sorted({v.size for k, v in g.items() if geo.kind(k) == geo.KIND_CELL})
    assert cells == [27, 36, 48, 64]


@pytest.mark.parametrize("n", [8, 16])
def test_root_size_exact_mode(n):
    # eps = 0 (no skeletonization): the root keeps every DOF with a coordinate on
    # the middle separator planes j = n/2: n^3 - (n-1)^3 of them.
    A = stencil.assemble(np.ones(n ** 3), 0.0, n)
    fac = hif.hif_factor(A, n, 4, 0.0)
    assert fac.root_size == n ** 3 - (n - 1) ** 3


@pytest.mark.parametrize("eps", [0.0, 1e-3])
def test_every_dof_eliminated_once(eps):
    n = 16
    rng = np.random.default_rng(7)
    A = stencil.assemble(10.0 ** rng.uniform(-1, 1, n ** 3), 0.0, n)
    fac = hif.hif_factor(A, n, 4, eps)
    parts = []
    for r in fac.records:
        parts.append(r.I if isinstance(r, hif.CellRecord) else r.Fc)
    parts.append(fac.root.S)
    allidx = np.concatenate(parts)
    assert allidx.size == n ** 3
    assert np.array_equal(np.sort(allidx), np.arange(n ** 3))


@pytest.mark.parametrize("n,m", [(8, 4), (16, 4), (32, 4), (12, 3)])
def test_periodic_group_counts_closed_form(n, m):
    # periodic grid: every multiple of s is a separator (each cell owns its
    # first frame, §2.1), so c^3 cells, 3c^3 faces, 3c^3 edges, c^3 vertices
    L = geo.num_levels(n, m)
    for level in range(L):
        s = m << level
        c = n // s
        got = geo.count_groups(n, s, periodic=True)
        assert got == {geo.KIND_CELL: c ** 3, geo.KIND_FACE: 3 * c ** 3,
                       geo.KIND_EDGE: 3 * c ** 3, geo.KIND_VERTEX: c ** 3}


def test_periodic_closures_wrap():
    # the last cell's closure holds plane 0; a face on plane 0 lies between
    # the last cell and the first
    n, s = 16, 4
    ncode = 2 * (n // s)
    last = (ncode - 1, 1, 1)
    assert (0, 1, 1) in geo.cell_closure(last, ncode)
    assert sorted(geo.adjacent_cells((0, 1, 1), ncode)) == [(1, 1, 1), (ncode - 1, 1, 1)]
    g = geo.group_active(np.arange(n ** 3), n, s, periodic=True)
    sizes = {geo.kind(k): v.size for k, v in g.items()}
    assert sizes == {0: 27, 1: 9, 2: 3, 3: 1}   # every group has the interior shape
