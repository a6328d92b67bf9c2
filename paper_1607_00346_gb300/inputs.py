"""Seeded synthetic inputs for the HIF workloads.

This module only draws random numbers; it holds none of the method's
arithmetic (no stencil, no factorisation).  Both the CPU oracle tests and the
GPU path take their inputs from here, so the two sides always see the same
arrays for the same seed.

Layout: a grid function on the n x n x n interior grid is a flat float64
array of length n**3 indexed ``j1 + n*j2 + n*n*j3`` (j1 fastest).  Several
right-hand sides are stored column after column (``N x nrhs``, each column
contiguous), i.e. a C-contiguous array of shape ``(nrhs, N)``.

Workloads (the paper uses synthetic coefficient fields only, §4):
  * constant coefficient ``a = 1`` (Example 1 uses a = 1),
  * high-contrast ``a = 10**U(lo, hi)`` drawn independently per grid point,
  * the Example 2 field (smoothed, thresholded uniform noise, {0.1, 1000})
    and the Example 3 checkerboard of 7-point blocks ({1000, 0.1}),
  * right-hand sides / test vectors with iid standard normal entries
    (the solve error of Table 2 uses a Gaussian random vector).
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 20260101


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(int(seed))


def coeff_constant(n: int, value: float = 1.0) -> np.ndarray:
    return np.full(n * n * n, float(value), dtype=np.float64)


def coeff_log_uniform(n: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """a_j = 10**u_j with u_j ~ U(lo, hi) iid per grid point."""
    u = rng(seed).uniform(lo, hi, size=n * n * n)
    return np.power(10.0, u)


def coeff_blurred_quantized(n: int, seed: int, sigma: float = 1.0, lo: float = 0.1,
                            hi: float = 1000.0) -> np.ndarray:
    """The paper's Example 2 field (§4): iid U(0,1) per grid point, smoothed
    by an isotropic Gaussian of standard deviation `sigma` grid spacings
    (periodic wrap, the paper's domain is periodic), then `lo` where the
    smoothed value is <= 0.5 and `hi` elsewhere."""
    from scipy import ndimage
    u = rng(seed).uniform(0.0, 1.0, size=(n, n, n))
    s = ndimage.gaussian_filter(u, sigma=sigma, mode="wrap")
    return np.where(s <= 0.5, lo, hi).reshape(-1)


def coeff_checkerboard(n: int, block: int = 7, lo: float = 0.1, hi: float = 1000.0) -> np.ndarray:
    """The paper's Example 3 field (§4): `hi` where the sum of the block
    indices floor(j_d / block) is even, `lo` where it is odd (j_d the 0-based
    grid index along dimension d)."""
    j = np.arange(n) // block
    s = j[:, None, None] + j[None, :, None] + j[None, None, :]
    return np.where(s % 2 == 0, hi, lo).astype(np.float64).reshape(-1)


def normal_rhs(n: int, nrhs: int, seed: int) -> np.ndarray:
    """nrhs iid N(0,1) grid functions, shape (nrhs, n**3) (columns contiguous)."""
    return rng(seed).standard_normal(size=(nrhs, n * n * n))


def workload(name: str):
    """Named workloads with their sizes; returns a dict of plain parameters.

    Every array is produced by the functions above from the stated seed.
    """
    table = {
        # 16^3 Laplacian, a = 1, b = 0, eps = 1e-6, one N(0,1) rhs
        "laplace16": dict(n=16, m=4, a=("const", 1.0), b=0.0, eps=1e-6,
                          nrhs=1, seed=SEED_BASE + 0),
        # 64^3, a = 10^U(-1,1), b = 0, eps 1e-4 / 1e-6, 8 rhs
        "contrast64": dict(n=64, m=4, a=("logu", -1.0, 1.0), b=0.0, eps=1e-6,
                           nrhs=8, seed=SEED_BASE + 1),
        # 128^3, a = 10^U(-1,1), b = 0.1, eps = 1e-6
        "contrast128": dict(n=128, m=4, a=("logu", -1.0, 1.0), b=0.1,
                            eps=1e-6, nrhs=1, seed=SEED_BASE + 2),
        # 256^3, a = 10^U(-3,3), b = 0, eps = 1e-4
        "contrast256": dict(n=256, m=4, a=("logu", -3.0, 3.0), b=0.0,
                            eps=1e-4, nrhs=1, seed=SEED_BASE + 4),
        # the paper's Example 2 field at 64^3 (b = 0.1, eps = 1e-5)
        "example2_64": dict(n=64, m=4, a=("blur", 1.0), b=0.1, eps=1e-5,
                            nrhs=1, seed=SEED_BASE + 5),
        # the paper's Example 3 checkerboard at 64^3 (b = 0.1, eps = 1e-4)
        "example3_64": dict(n=64, m=4, a=("checker", 7), b=0.1, eps=1e-4,
                            nrhs=1, seed=SEED_BASE + 6),
    }
    return dict(table[name])


def make_coeff(n: int, spec, seed: int) -> np.ndarray:
    if spec[0] == "const":
        return coeff_constant(n, spec[1])
    if spec[0] == "logu":
        return coeff_log_uniform(n, spec[1], spec[2], seed)
    if spec[0] == "blur":
        return coeff_blurred_quantized(n, seed, sigma=spec[1])
    if spec[0] == "checker":
        return coeff_checkerboard(n, block=spec[1])
    raise ValueError(f"unknown coefficient spec {spec!r}")
