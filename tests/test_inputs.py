"""Seeded input generators: determinism, value sets and the closed-form
checkerboard of the paper's Example 3 (§4)."""
import numpy as np

from paper_1607_00346_gb300 import inputs


def test_checkerboard_closed_form():
    n = 20
    a = inputs.coeff_checkerboard(n).reshape(n, n, n)   # [j3, j2, j1]
    for j3, j2, j1 in [(0, 0, 0), (0, 0, 7), (0, 7, 7), (7, 7, 7), (13, 14, 6), (19, 0, 3)]:
        even = (j1 // 7 + j2 // 7 + j3 // 7) % 2 == 0
        assert a[j3, j2, j1] == (1000.0 if even else 0.1)


def test_blurred_field_two_values_and_seeded():
    a = inputs.coeff_blurred_quantized(24, 5)
    b = inputs.coeff_blurred_quantized(24, 5)
    c = inputs.coeff_blurred_quantized(24, 6)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    vals, counts = np.unique(a, return_counts=True)
    assert list(vals) == [0.1, 1000.0]
    # the smoothed noise has mean 1/2, so the threshold splits it about evenly
    assert 0.35 < counts[1] / a.size < 0.65


def test_blurred_field_is_spatially_correlated():
    # smoothing makes neighbours agree far more often than iid labels would (1/2)
    n = 32
    a = inputs.coeff_blurred_quantized(n, 11).reshape(n, n, n)
    agree = np.mean(a[:, :, 1:] == a[:, :, :-1])
    assert agree > 0.7


def test_workload_table_builds_every_field():
    for name in ("laplace16", "contrast64", "example2_64", "example3_64"):
        w = inputs.workload(name)
        a = inputs.make_coeff(8, w["a"], w["seed"])
        assert a.shape == (512,) and np.all(a > 0)
