"""GPU path vs the CPU oracle on the same seeded inputs (through the C ABI).

Tolerances:
  * eps = 0 (exact multifrontal elimination): F^{-1} f agrees with the oracle
    and with a dense Cholesky solve to 1e-10 relative in FP64;
  * eps > 0: the solve error e_s = ||x - F^{-1} A x|| / ||x|| of the GPU factor
    is within 2x the oracle's (+ an FP64 rounding floor of 1e-12): the two
    sides may pick different, equally valid skeletons on ties;
  * PCG: relative residual <= 1e-10 (checked again on the CPU with the
    oracle's operator), solution vs the dense solve within 1e-8.
"""
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


def _coeff(n, seed, lo=-1.0, hi=1.0):
    return inputs.coeff_log_uniform(n, lo, hi, seed)


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _gpu_apply(h, f):
    fd = _dev(f)
    ud = torch.empty_like(fd)
    h.apply(fd, ud)
    torch.cuda.synchronize()
    return ud.cpu().numpy()


@pytest.mark.parametrize("n,m,b", [(8, 4, 0.0), (16, 4, 0.3), (12, 3, 0.0), (20, 5, 0.1)])
def test_exact_mode_matches_oracle_and_dense(H, n, m, b):
    a = _coeff(n, 100 + n)
    A = stencil.assemble(a, b, n)
    f = inputs.normal_rhs(n, 3, 200 + n)
    h = H.factor(n, m, _dev(a), b_const=b, eps=0.0)
    u = _gpu_apply(h, f)
    ref = sla.cho_solve(sla.cho_factor(A.toarray()), f.T).T
    assert np.linalg.norm(u - ref) <= 1e-10 * np.linalg.norm(ref)
    fac = ohif.hif_factor(A, n, m, 0.0)
    uo = ohif.hif_apply(fac, f)
    assert np.linalg.norm(u - uo) <= 1e-10 * np.linalg.norm(uo)
    st = h.stats()
    assert st["root_size"] == fac.root_size == n ** 3 - (n - 1) ** 3


def _es_gpu(h, A, x):
    return np.linalg.norm(x - _gpu_apply(h, A @ x)) / np.linalg.norm(x)


@pytest.mark.parametrize("n,eps,lo,hi", [(16, 1e-6, 0.0, 0.0), (16, 1e-3, -1.0, 1.0),
                                         (32, 1e-4, -1.0, 1.0), (32, 1e-6, -1.0, 1.0)])
def test_skeletonized_solve_error_within_2x_oracle(H, n, eps, lo, hi):
    a = inputs.coeff_constant(n) if lo == hi else _coeff(n, 300 + n, lo, hi)
    A = stencil.assemble(a, 0.0, n)
    x = inputs.normal_rhs(n, 1, 400 + n)[0]
    h = H.factor(n, 4, _dev(a), eps=eps)
    es_g = _es_gpu(h, A, x)
    fac = ohif.hif_factor(A, n, 4, eps, check=False)
    es_o = krylov.solve_error(A, fac, x)
    assert es_g <= 2.0 * es_o + 1e-12, (es_g, es_o)
    st = h.stats()
    # both sides compress: root well below the exact-mode size, close to the oracle's
    assert st["root_size"] <= n ** 3 - (n - 1) ** 3
    assert abs(st["root_size"] - fac.root_size) <= 0.1 * fac.root_size + 8


def test_laplace16_config(H):
    # 16^3, a = 1, b = 0, eps = 1e-6, one N(0,1) right-hand side
    w = inputs.workload("laplace16")
    n = w["n"]
    a = inputs.make_coeff(n, w["a"], w["seed"])
    f = inputs.normal_rhs(n, w["nrhs"], w["seed"] + 1)
    A = stencil.assemble(a, w["b"], n)
    h = H.factor(n, w["m"], _dev(a), b_const=w["b"], eps=w["eps"])
    u = torch.zeros(f.shape, dtype=torch.float64, device="cuda")
    its, rel = h.solve(_dev(f), u)
    uc = u.cpu().numpy()
    assert rel[0] <= 1e-10 and its[0] <= 5
    r = f[0] - A @ uc[0]
    assert np.linalg.norm(r) <= 1.0000001e-10 * np.linalg.norm(f[0])
    ref = sla.cho_solve(sla.cho_factor(A.toarray()), f[0])
    assert np.linalg.norm(uc[0] - ref) <= 1e-8 * np.linalg.norm(ref)


@pytest.mark.parametrize("precision", [0, 1])
def test_pcg_multi_rhs(H, precision):
    n = 32
    a = _coeff(n, 501)
    A = stencil.assemble(a, 0.1, n)
    f = inputs.normal_rhs(n, 4, 502)
    h = H.factor(n, 4, _dev(a), b_const=0.1, eps=1e-6, precision=precision)
    u = torch.zeros(f.shape, dtype=torch.float64, device="cuda")
    its, rel = h.solve(_dev(f), u)
    uc = u.cpu().numpy()
    for c in range(4):
        assert rel[c] <= 1e-10
        assert np.linalg.norm(f[c] - A @ uc[c]) <= 1.0000001e-10 * np.linalg.norm(f[c])
    assert max(its) <= (6 if precision == 0 else 25)
    # against the oracle's own PCG (FP64 factor, same eps): both at 1e-10 residual
    fac = ohif.hif_factor(A, n, 4, 1e-6, check=False)
    uo, ito, _ = krylov.pcg(A, fac, f[1], tol=1e-12)
    assert np.linalg.norm(uc[1] - uo) <= 1e-8 * np.linalg.norm(uo)


@pytest.mark.parametrize("precision", [0, 1])
def test_multi_rhs_apply_is_bitwise_per_column(H, precision):
    # the apply's mat-vecs take right-hand sides in blocks of 16, 8, 4, 2 and 1
    # (one read of the factor per block) with the same arithmetic for every
    # column in any block: a 23-column apply (16 + 4 + 2 + 1) equals 23
    # one-column applies bit for bit
    n = 16
    a = _coeff(n, 981)
    f = inputs.normal_rhs(n, 23, 982)
    h = H.factor(n, 4, _dev(a), b_const=0.1, eps=1e-6, precision=precision)
    ub = _gpu_apply(h, f)
    for c in range(23):
        uc = _gpu_apply(h, f[c:c + 1])
        assert np.array_equal(ub[c], uc[0]), c
    h.close()


def test_residual_matches_oracle_operator(H):
    n = 16
    a = _coeff(n, 601)
    A = stencil.assemble(a, 0.25, n)
    h = H.factor(n, 4, _dev(a), b_const=0.25, eps=0.0)
    f, u = inputs.normal_rhs(n, 2, 602), inputs.normal_rhs(n, 2, 603)
    r = torch.empty(f.shape, dtype=torch.float64, device="cuda")
    h.residual(_dev(f), _dev(u), r)
    ref = f - (A @ u.T).T
    assert np.allclose(r.cpu().numpy(), ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_host_pointers_and_in_place(H):
    n = 16
    a = _coeff(n, 701)
    h = H.factor(n, 4, a, eps=1e-4)                  # host array in
    f = inputs.normal_rhs(n, 1, 702)
    u_host = np.zeros_like(f)
    h.apply(f, u_host)                               # host in, host out
    u_dev = _gpu_apply(h, f)
    assert np.array_equal(u_host, u_dev)
    fd = _dev(f)
    h.apply(fd, fd)                                  # in place
    assert np.array_equal(fd.cpu().numpy(), u_dev)


def test_deterministic_reruns(H):
    n = 32
    a = _coeff(n, 801)
    f = inputs.normal_rhs(n, 2, 802)
    u1 = _gpu_apply(H.factor(n, 4, _dev(a), eps=1e-4, precision=1), f)
    u2 = _gpu_apply(H.factor(n, 4, _dev(a), eps=1e-4, precision=1), f)
    assert np.array_equal(u1, u2)


def test_fp32_factor_preconditioner_quality(H):
    n = 32
    a = _coeff(n, 901)
    A = stencil.assemble(a, 0.0, n)
    x = inputs.normal_rhs(n, 1, 902)[0]
    h64 = H.factor(n, 4, _dev(a), eps=1e-6, precision=0)
    h32 = H.factor(n, 4, _dev(a), eps=1e-6, precision=1)
    e64, e32 = _es_gpu(h64, A, x), _es_gpu(h32, A, x)
    assert e64 < 1e-5
    assert e32 < 1e-2


def test_invalid_coefficients(H):
    n = 8
    a = np.ones(n ** 3)
    a[17] = -1.0
    with pytest.raises(H.HifError) as e:
        H.factor(n, 4, _dev(a))
    assert e.value.status == 1
    a[17] = np.nan
    with pytest.raises(H.HifError):
        H.factor(n, 4, _dev(a))
    # the context is still usable afterwards
    h = H.factor(n, 4, _dev(np.ones(n ** 3)), eps=0.0)
    assert h.stats()["root_size"] == n ** 3 - (n - 1) ** 3


@pytest.mark.parametrize("field,n,eps", [("blur", 32, 1e-5), ("checker", 32, 1e-4)])
def test_paper_example_fields_within_2x_oracle(H, field, n, eps):
    # the paper's Example 2 (smoothed thresholded noise) and Example 3
    # (checkerboard) coefficient fields, b = 0.1: contrast 10^4
    a = (inputs.coeff_blurred_quantized(n, 610 + n) if field == "blur"
         else inputs.coeff_checkerboard(n))
    A = stencil.assemble(a, 0.1, n)
    x = inputs.normal_rhs(n, 1, 620 + n)[0]
    h = H.factor(n, 4, _dev(a), b_const=0.1, eps=eps)
    es_g = _es_gpu(h, A, x)
    fac = ohif.hif_factor(A, n, 4, eps, check=False)
    es_o = krylov.solve_error(A, fac, x)
    assert es_g <= 2.0 * es_o + 1e-12, (es_g, es_o)
    f = inputs.normal_rhs(n, 1, 630 + n)
    u = torch.zeros(f.shape, dtype=torch.float64, device="cuda")
    its, rel = h.solve(_dev(f), u)
    r = f[0] - A @ u.cpu().numpy()[0]
    assert rel[0] <= 1e-10 and np.linalg.norm(r) <= 1.0000001e-10 * np.linalg.norm(f[0])


def test_graph_replayed_apply_is_bitwise_the_launched_one(H):
    # the apply sweeps captured in a CUDA graph run the same kernels in the
    # same order as the launched sweeps: identical results, also on replay
    n = 32
    a = _coeff(n, 951)
    f = inputs.normal_rhs(n, 3, 952)
    hg = H.factor(n, 4, _dev(a), eps=1e-6, precision=1, use_graphs=True)
    hl = H.factor(n, 4, _dev(a), eps=1e-6, precision=1, use_graphs=False)
    ug1 = _gpu_apply(hg, f)
    ug2 = _gpu_apply(hg, f)          # replay of the captured graph
    ul = _gpu_apply(hl, f)
    assert np.array_equal(ug1, ul) and np.array_equal(ug2, ul)
    u1 = torch.zeros(f.shape, dtype=torch.float64, device="cuda")
    u2 = torch.zeros(f.shape, dtype=torch.float64, device="cuda")
    its1, _ = hg.solve(_dev(f), u1)
    its2, _ = hl.solve(_dev(f), u2)
    torch.cuda.synchronize()
    assert its1 == its2 and torch.equal(u1, u2)


@pytest.mark.parametrize("precision", [0, 1])
def test_saved_and_loaded_factor_is_bitwise_the_same(H, tmp_path, precision):
    n = 16
    a = _coeff(n, 971)
    f = inputs.normal_rhs(n, 2, 972)
    h = H.factor(n, 4, _dev(a), b_const=0.1, eps=1e-6, precision=precision)
    path = str(tmp_path / "f.hiff")
    h.save(path)
    h2 = H.load_factor(path)
    assert np.array_equal(_gpu_apply(h, f), _gpu_apply(h2, f))
    st, st2 = h.stats(), h2.stats()
    assert st["root_size"] == st2["root_size"] and st["stored_entries"] == st2["stored_entries"]
    u1 = torch.zeros(f.shape, dtype=torch.float64, device="cuda")
    u2 = torch.zeros(f.shape, dtype=torch.float64, device="cuda")
    its1, _ = h.solve(_dev(f), u1)
    its2, _ = h2.solve(_dev(f), u2)
    torch.cuda.synchronize()
    assert its1 == its2 and torch.equal(u1, u2)


def test_load_rejects_inconsistent_factor_files(H, tmp_path):
    # a file whose sizes are all valid but whose contents disagree with each
    # other (a stale work stride, a gather index outside the grid) is refused
    # before any kernel could read out of bounds
    import ctypes
    n = 8
    h = H.factor(n, 4, _dev(_coeff(n, 990)), eps=1e-6, precision=1)
    path = tmp_path / "f.hiff"
    h.save(str(path))
    raw = bytearray(path.read_bytes())
    head = 4 + 3 * 4                                   # magic, version, two struct sizes
    scalars = 4 * 4 + 8 + 4                            # n, m, L, precision, eps, bc
    ws_off = head + scalars + ctypes.sizeof(H.Options) + ctypes.sizeof(H.Stats)
    N = n ** 3
    stale = bytearray(raw)
    ws = int.from_bytes(stale[ws_off:ws_off + 8], "little")
    stale[ws_off:ws_off + 8] = (ws + 2).to_bytes(8, "little")
    (tmp_path / "stale.hiff").write_bytes(stale)
    with pytest.raises(H.HifError) as e:
        H.load_factor(str(tmp_path / "stale.hiff"))
    assert e.value.status == 1 and "work stride" in str(e.value)
    # first stage's gather list: after the operator arrays (byte count + data
    # each), the stage count and the stage's six scalars, and its byte count
    idx_off = ws_off + 8 + (8 + 24 * N) + (8 + 8 * N) + 8 + (4 + 4 + 4 * 8) + 8
    bad = bytearray(raw)
    bad[idx_off:idx_off + 4] = (N + 5).to_bytes(4, "little")
    (tmp_path / "bad_index.hiff").write_bytes(bad)
    with pytest.raises(H.HifError) as e:
        H.load_factor(str(tmp_path / "bad_index.hiff"))
    assert e.value.status == 1 and "gather index" in str(e.value)
    # the untouched file still loads and applies exactly as the original
    h2 = H.load_factor(str(path))
    f = inputs.normal_rhs(n, 1, 991)
    assert np.array_equal(_gpu_apply(h, f), _gpu_apply(h2, f))


def test_measured_peaks_are_plausible(H):
    # hif_measure_peaks times FMA and tensor-core loops on this GPU; the
    # roofline denominators of the benchmark come from it
    p = H.measure_peaks()
    assert p["sm_count"] > 0 and p["sm_clock_khz"] > 0
    assert p["fp32_fma_tflops"] > 5 * p["fp64_fma_tflops"] > 0
    assert p["tf32_mma_tflops"] > 2 * p["fp32_fma_tflops"]
    assert p["bf16_mma_tflops"] > 1.5 * p["tf32_mma_tflops"]
    # FMA: at most 128 lanes x 2 flops x clock per SM
    assert p["fp32_fma_tflops"] <= 1.05 * p["sm_count"] * 256 * p["sm_clock_khz"] * 1e3 / 1e12


def test_fp64_retry_of_fronts_flagged_by_pivot_growth(H):
    # contrast 10^8 (a = 10^U(-4,4)), FP32 factor: fronts whose Cholesky loses
    # most of a pivot to cancellation (A_jj / d_j > retry_growth) are
    # refactored in double.  The retried factor must still meet the parity
    # bounds (PCG solution equal to the oracle's to 1e-8, e_s no worse than
    # the factor without retries), and forcing retries (a small threshold)
    # may only make the factor better.
    n, eps = 32, 1e-6
    a = _coeff(n, 1201, -4.0, 4.0)
    A = stencil.assemble(a, 0.0, n)
    x = inputs.normal_rhs(n, 1, 1202)[0]
    f = inputs.normal_rhs(n, 1, 1203)
    out = {}
    for g in (0.0, 1e5, 1e2):
        try:
            h = H.factor(n, 4, _dev(a), eps=eps, precision=1, retry_growth=g)
        except H.HifError as e:          # without retries FP32 may break down
            assert g == 0.0 and e.status == 3, e
            out[g] = None
            continue
        es = _es_gpu(h, A, x)
        u = torch.zeros(f.shape, dtype=torch.float64, device="cuda")
        its, rel = h.solve(_dev(f), u, check=False)
        out[g] = (h.stats()["retried_fronts"], es, its[0], rel[0], u.cpu().numpy()[0])
        h.close()
    print("\n[retry] " + "; ".join(f"growth {g:g}: " + ("NOT_SPD" if v is None else
          f"retried {v[0]}, e_s {v[1]:.2e}, PCG {v[2]} its relres {v[3]:.1e}")
          for g, v in out.items()))
    assert out[1e2][0] > 0
    fac = ohif.hif_factor(A, n, 4, eps, check=False)
    uo, _, _ = krylov.pcg(A, fac, f[0], tol=1e-12)
    for g in (1e5, 1e2):
        retried, es, its, rel, u = out[g]
        assert rel <= 1e-10, (g, rel)
        assert np.linalg.norm(u - uo) <= 1e-8 * np.linalg.norm(uo), g
    if out[0.0] is not None:
        assert out[1e2][1] <= 1.5 * out[0.0][1], (out[1e2][1], out[0.0][1])


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_apply_and_solve_are_bitwise_the_single_ones(H, precision):
    # factors of different grids (and leaf sizes), different numbers of
    # right-hand sides: hif_apply_batch / hif_solve_batch run their sweeps in
    # shared launches, and every factor's result must be bit for bit its own
    # hif_apply / hif_solve
    grids = [(16, 4, 3), (24, 3, 1), (32, 4, 5), (8, 4, 17)]
    hs, fs = [], []
    for k, (n, m, nr) in enumerate(grids):
        a = _coeff(n, 1600 + k)
        hs.append(H.factor(n, m, _dev(a), b_const=0.05 * k, eps=1e-6, precision=precision))
        fs.append(inputs.normal_rhs(n, nr, 1610 + k))
    fd = [_dev(f) for f in fs]
    us = [torch.full_like(f, float("nan")) for f in fd]
    H.apply_batch(hs, fd, us)
    torch.cuda.synchronize()
    for h, f, u in zip(hs, fd, us):
        ref = torch.empty_like(f)
        h.apply(f, ref)
        torch.cuda.synchronize()
        assert torch.equal(u, ref)
    # host arrays in the batch too
    uh = [np.zeros_like(f) for f in fs]
    H.apply_batch(hs, fs, uh)
    for u, ub in zip(uh, us):
        assert np.array_equal(u, ub.cpu().numpy())
    us = [torch.zeros_like(f) for f in fd]
    res = H.solve_batch(hs, fd, us)
    torch.cuda.synchronize()
    for h, f, u, (its, rel) in zip(hs, fd, us, res):
        ref = torch.zeros_like(f)
        its1, rel1 = h.solve(f, ref)
        torch.cuda.synchronize()
        assert torch.equal(u, ref) and its == its1 and rel == rel1
        assert max(rel) <= 1e-10
    with pytest.raises(H.HifError):
        H.apply_batch([hs[0], hs[0]], [fd[0], fd[0]], [us[0], us[1]])
    for h in hs:
        h.close()
