"""The autotuner (hif_autotune): launch shapes per size bucket chosen by
timing, among shapes that leave every result bit unchanged.

At 64^3 (contrast64, FP32 factor, eps 1e-6) one tuning factorization fills
the table (cluster-ID buckets measured in place, tensor-core product buckets
replayed); a factorization with the tuned table must then be bitwise the one
with the built-in rules: the same active sets after every level, the same
apply results and the same PCG solution.  A written table loads back.
"""
import numpy as np
import pytest

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


def test_tuned_factor_is_bitwise_the_built_in_one(H, tmp_path):
    w = inputs.workload("contrast64")
    n, m = w["n"], w["m"]
    a = _dev(inputs.make_coeff(n, w["a"], w["seed"]))
    f = _dev(inputs.normal_rhs(n, 3, w["seed"] + 1))

    def run():
        h = H.factor(n, m, a, eps=1e-6, precision=H.PREC_FP32)
        act = [h.active(l) for l in range(4)]
        y = torch.empty_like(f)
        h.apply(f, y)
        u = torch.zeros_like(f)
        its, _ = h.solve(f, u)
        torch.cuda.synchronize()
        h.close()
        return act, y.cpu().numpy(), u.cpu().numpy(), its

    H.autotune_clear()
    ref = run()
    path = str(tmp_path / "tune.txt")
    table = H.autotune(n, m, a, eps=1e-6, precision=H.PREC_FP32, path=path, force=True)
    print("\n[autotune 64^3]\n" + table)
    lines = [l.split() for l in table.splitlines() if l and not l.startswith("#")]
    assert any(l[0] == "id" for l in lines) and any(l[0] == "gemm" for l in lines)
    tuned = run()
    for x, y in zip(ref[0], tuned[0]):
        assert np.array_equal(x, y)
    assert np.array_equal(ref[1], tuned[1]) and np.array_equal(ref[2], tuned[2])
    assert ref[3] == tuned[3]
    # the file loads back into the same table; without force it is not re-measured
    def entries(t):   # the table without its comment lines (measured times)
        return [l for l in t.splitlines() if l and not l.startswith("#")]

    H.autotune_clear()
    H.autotune_load(path)
    assert entries(H.autotune_table()) == entries(table)
    H.autotune_clear()
    assert entries(H.autotune(n, m, a, eps=1e-6, precision=H.PREC_FP32, path=path)) == entries(table)
    H.autotune_clear()
