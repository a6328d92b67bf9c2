"""Oracle runs for the GPU parity tests, in processes of their own.

The 64^3 factorizations take a minute or two each on the host, so the tests
start them in spawned worker processes (never forked after a GPU call) and
take back only what the comparisons need.  Test infrastructure only.
"""
from __future__ import annotations

import numpy as np


def oracle_contrast64(eps: float) -> dict:
    """The oracle on the contrast64 workload (n = 64, m = 4, a = 10^U(-1,1),
    b = 0) at this eps: F^{-1} A x for a seeded Gaussian x, its solve error,
    the PCG solution of A u = f (first workload right-hand side) to 1e-12, the
    active set after every level and every ID's decision."""
    from oracle import hif as ohif
    from oracle import krylov, stencil
    from paper_1607_00346_gb300 import inputs

    w = inputs.workload("contrast64")
    n, m, seed = w["n"], w["m"], w["seed"]
    a = inputs.make_coeff(n, w["a"], seed)
    A = stencil.assemble(a, w["b"], n)
    fac = ohif.hif_factor(A, n, m, eps, check=False, record=True)
    x = inputs.normal_rhs(n, 1, seed + 9)[0]
    y = ohif.hif_apply(fac, A @ x)
    es = float(np.linalg.norm(x - y) / np.linalg.norm(x))
    f = inputs.normal_rhs(n, 1, seed + 1)[0]
    u, its, hist = krylov.pcg(A, fac, f, tol=1e-12)
    ids = [(int(l), int(k), F.astype(np.int32), S.astype(np.int32), float(mg))
           for (l, k, F, S, mg) in fac.ids]
    return dict(eps=eps, y=y, es=es, u=u, pcg_iters=int(its), root=fac.root_size,
                ranks=list(fac.ranks), active=[a_.astype(np.int32) for a_ in fac.active],
                ids=ids)
