"""hif_apply_noalloc: the apply for callers that must not allocate device memory.

Some callers cannot allocate device memory at apply time: a serving process
that reserved all of its memory up front, or code that runs where calling the
CUDA allocator is not allowed.  hif_apply_noalloc gives them u = F^{-1} f with
the work space taken from the library's fixed 32 MiB device array instead of
buffers allocated on the handle.  Here it is checked against hif_apply on the
same handle, through the C ABI, on two calls in a row (the array keeps the
previous call's contents), and its refusals are checked: host pointers and
requests larger than the array.  Both entry points run the same kernels in
the same order on the same factor, so the results must agree bit for bit.

This file sorts last so that a run stopping at its first failure has already
run every other test.
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


@pytest.mark.parametrize("n,precision,nrhs", [(16, 0, 1), (32, 1, 2), (64, 0, 1)])
def test_noalloc_apply_matches_apply_twice(H, n, precision, nrhs):
    a = inputs.coeff_log_uniform(n, -1.0, 1.0, 1000 + n)
    h = H.factor(n, 4, _dev(a), b_const=0.1, eps=1e-6, precision=precision)
    for call in range(2):
        f = _dev(inputs.normal_rhs(n, nrhs, 2000 + 10 * n + call))
        u_ref = torch.empty_like(f)
        h.apply(f, u_ref)
        u = torch.full_like(f, float("nan"))
        h.apply_noalloc(f, u)
        torch.cuda.synchronize()
        assert torch.isfinite(u).all()
        assert torch.equal(u, u_ref), call
    h.close()


def test_noalloc_apply_refuses_what_it_cannot_do(H):
    n = 16
    h = H.factor(n, 4, _dev(np.ones(n ** 3)), eps=1e-6)
    f = inputs.normal_rhs(n, 1, 3001)
    with pytest.raises(H.HifError) as e:
        h.apply_noalloc(f, np.zeros_like(f))          # host arrays would need staging
    assert e.value.status == 1
    h.close()
    # 64^3 in FP64 with 8 right-hand sides needs far more than the fixed 32 MiB
    n = 64
    h = H.factor(n, 4, _dev(np.ones(n ** 3)), eps=1e-6, precision=0)
    f = _dev(inputs.normal_rhs(n, 8, 3002))
    with pytest.raises(H.HifError) as e:
        h.apply_noalloc(f, torch.empty_like(f))
    assert e.value.status == 1 and "bytes" in str(e.value)
    # the handle still works afterwards
    u = torch.empty_like(f[:1].contiguous())
    h.apply_noalloc(f[:1].contiguous(), u)
    u_ref = torch.empty_like(u)
    h.apply(f[:1].contiguous(), u_ref)
    torch.cuda.synchronize()
    assert torch.equal(u, u_ref)
    h.close()
