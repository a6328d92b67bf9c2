"""The periodic grid on the GPU (the paper's own setting, §2.1 and §4) against
the oracle's periodic operator and factorization, through the C ABI.

  * eps = 0: F^{-1} f equals a dense Cholesky solve and the oracle's exact
    factorization to 1e-10 (FP64); the root keeps n^3 - (n-2)^3 points (the
    separator planes of the top level);
  * residual r = f - A u equal to the oracle's periodic operator;
  * eps > 0: the solve error e_s within 2x the oracle's (FP64);
  * the paper's Example 1 at 32^3 (a = 1, b = 0.1 against the stencil
    without its 1/h^2, i.e. b = 0.1 n^2 here; eps = 1e-3, m = 4;
    tests/golden/example1_periodic_32.txt): the top-level point count of the
    printed table and e_s inside its printed range, in FP64 and FP32.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import hif as ohif
from oracle import krylov, stencil
from paper_1607_00346_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_00346_gb300 import build, hif
    build.build_library()
    hif.load()
    return hif


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _apply(h, f):
    fd = _dev(f)
    ud = torch.empty_like(fd)
    h.apply(fd, ud)
    torch.cuda.synchronize()
    return ud.cpu().numpy()


@pytest.mark.parametrize("n,m,b", [(8, 4, 1.0), (12, 3, 5.0), (16, 4, 20.0)])
def test_periodic_exact_mode_matches_dense_and_oracle(H, n, m, b):
    a = inputs.coeff_log_uniform(n, -1.0, 1.0, 1300 + n)
    A = stencil.assemble(a, b, n, periodic=True)
    f = inputs.normal_rhs(n, 2, 1310 + n)
    h = H.factor(n, m, _dev(a), b_const=b, eps=0.0, periodic=True)
    u = _apply(h, f)
    ref = sla.cho_solve(sla.cho_factor(A.toarray()), f.T).T
    assert np.linalg.norm(u - ref) <= 1e-10 * np.linalg.norm(ref)
    fac = ohif.hif_factor(A, n, m, 0.0, periodic=True)
    assert np.linalg.norm(u - ohif.hif_apply(fac, f)) <= 1e-10 * np.linalg.norm(ref)
    assert h.stats()["root_size"] == fac.root_size == n ** 3 - (n - 2) ** 3
    # the residual with the handle's operator is the oracle's operator
    uu = inputs.normal_rhs(n, 2, 1320 + n)
    r = torch.empty(f.shape, dtype=torch.float64, device="cuda")
    h.residual(_dev(f), _dev(uu), r)
    rr = f - (A @ uu.T).T
    assert np.allclose(r.cpu().numpy(), rr, rtol=0, atol=1e-12 * np.abs(rr).max())


@pytest.mark.parametrize("n,eps", [(16, 1e-3), (32, 1e-4), (32, 1e-6)])
def test_periodic_solve_error_within_2x_oracle(H, n, eps):
    a = inputs.coeff_log_uniform(n, -1.0, 1.0, 1400 + n)
    b = 0.1 * n * n
    A = stencil.assemble(a, b, n, periodic=True)
    x = inputs.normal_rhs(n, 1, 1410 + n)[0]
    h = H.factor(n, 4, _dev(a), b_const=b, eps=eps, periodic=True)
    es_g = float(np.linalg.norm(x - _apply(h, A @ x)) / np.linalg.norm(x))
    fac = ohif.hif_factor(A, n, 4, eps, check=False, periodic=True)
    es_o = krylov.solve_error(A, fac, x)
    print(f"\n[periodic] n={n} eps={eps}: e_s gpu {es_g:.3e} oracle {es_o:.3e}, "
          f"root gpu {h.stats()['root_size']} oracle {fac.root_size}")
    assert es_g <= 2.0 * es_o + 1e-12, (es_g, es_o)
    assert abs(h.stats()["root_size"] - fac.root_size) <= 0.02 * fac.root_size
    f = inputs.normal_rhs(n, 1, 1420 + n)
    u = torch.zeros(f.shape, dtype=torch.float64, device="cuda")
    its, rel = h.solve(_dev(f), u)
    r = f[0] - A @ u.cpu().numpy()[0]
    assert rel[0] <= 1e-10 and np.linalg.norm(r) <= 1.0000001e-10 * np.linalg.norm(f[0])


def _golden_example1():
    path = os.path.join(os.path.dirname(__file__), "golden", "example1_periodic_32.txt")
    g = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()
        g[k] = float(v)
    return g


@pytest.mark.parametrize("precision", [0, 1])
def test_periodic_example1_matches_the_papers_table(H, precision):
    g = _golden_example1()
    n, m = int(g["n"]), int(g["m"])
    b = g["b_over_stencil"] * n * n
    A = stencil.assemble(np.ones(n ** 3), b, n, periodic=True)
    h = H.factor(n, m, _dev(np.ones(n ** 3)), b_const=b, eps=g["eps"], precision=precision,
                 periodic=True)
    x = inputs.normal_rhs(n, 1, 1501)[0]
    es = float(np.linalg.norm(x - _apply(h, A @ x)) / np.linalg.norm(x))
    f = inputs.normal_rhs(n, 1, 1502)
    u = torch.zeros(f.shape, dtype=torch.float64, device="cuda")
    its, rel = h.solve(_dev(f), u)
    root = h.stats()["root_size"]
    print(f"\n[example1 periodic 32^3] precision {precision}: root {root} (paper {int(g['root_size'])}), "
          f"e_s {es:.3e} (paper {g['es_min']:.2e} .. {g['es_max']:.2e}), PCG {its[0]} its to {rel[0]:.1e}")
    assert root == int(g["root_size"])
    assert g["es_min"] <= es <= g["es_max"], es
    assert rel[0] <= 1e-10 and its[0] <= 10
