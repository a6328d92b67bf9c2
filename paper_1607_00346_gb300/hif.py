"""Python binding of the HIF C ABI (include/hif.h).

Argument marshalling only: every step of the factorization, the apply and the
solve runs in the CUDA library ``libhif.so``.  Arrays may be CUDA tensors
(passed by device pointer, on the tensor's device) or numpy arrays / CPU
tensors (passed by host pointer; the library copies them).  There is no CPU
fallback: without the built library every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

HIF_OK = 0
STATUS = {0: "HIF_OK", 1: "HIF_ERR_INVALID_ARG", 2: "HIF_ERR_OOM", 3: "HIF_ERR_NOT_SPD",
          4: "HIF_ERR_NO_CONVERGENCE", 5: "HIF_ERR_TIMEOUT", 6: "HIF_ERR_CUDA"}
PREC_FP64, PREC_FP32 = 0, 1


class HifError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("m", ctypes.c_int), ("bc", ctypes.c_int)]


class Options(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("precision", ctypes.c_int),
                ("use_graphs", ctypes.c_int), ("pcg_tol", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("tensor_cores", ctypes.c_int),
                ("retry_growth", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("m", ctypes.c_int), ("levels", ctypes.c_int),
                ("precision", ctypes.c_int), ("eps", ctypes.c_double),
                ("root_size", ctypes.c_int),
                ("active_after", ctypes.c_int64 * 16),
                ("fronts", (ctypes.c_int64 * 3) * 16),
                ("factor_seconds", ctypes.c_double),
                ("level_seconds", ctypes.c_double * 17),
                ("flops", ctypes.c_double),
                ("factor_bytes", ctypes.c_size_t),
                ("peak_bytes", ctypes.c_size_t),
                ("stored_entries", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int),
                ("apply_launches", ctypes.c_int),
                ("retried_fronts", ctypes.c_int64)]


_lib = None

# every symbol declared in include/hif.h
EXPORTS = ["hif_default_options", "hif_factor", "hif_apply", "hif_apply_noalloc",
           "hif_residual", "hif_solve",
           "hif_query_stats", "hif_predict_bytes", "hif_profile_begin", "hif_profile_end",
           "hif_destroy", "hif_last_error", "hif_version", "hif_save", "hif_load",
           "hif_measure_peaks", "hif_query_active", "hif_apply_batch", "hif_solve_batch",
           "hif_autotune", "hif_autotune_load", "hif_autotune_clear", "hif_autotune_table"]


class Peaks(ctypes.Structure):
    _fields_ = [("sm_count", ctypes.c_int), ("sm_clock_khz", ctypes.c_int),
                ("fp32_fma_tflops", ctypes.c_double), ("fp64_fma_tflops", ctypes.c_double),
                ("tf32_mma_tflops", ctypes.c_double), ("bf16_mma_tflops", ctypes.c_double),
                ("seconds", ctypes.c_double)]


class KernelProfile(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64),
                ("kernels", ctypes.c_int64), ("seconds", ctypes.c_double),
                ("flops", ctypes.c_double), ("bytes", ctypes.c_double)]


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libhif.so (built by ``build.build_library``); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"HIF CUDA library not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.hif_default_options.argtypes = [ctypes.POINTER(Options)]
    lib.hif_default_options.restype = None
    lib.hif_factor.argtypes = [ctypes.POINTER(Grid), vp, vp, d, ctypes.POINTER(Options), vp,
                               ctypes.POINTER(vp)]
    lib.hif_factor.restype = i
    lib.hif_apply.argtypes = [vp, vp, vp, i, vp]
    lib.hif_apply.restype = i
    lib.hif_apply_noalloc.argtypes = [vp, vp, vp, i, vp]
    lib.hif_apply_noalloc.restype = i
    lib.hif_residual.argtypes = [vp, vp, vp, vp, i, vp]
    lib.hif_residual.restype = i
    lib.hif_solve.argtypes = [vp, vp, vp, i, vp, ctypes.POINTER(ctypes.c_int),
                              ctypes.POINTER(ctypes.c_double)]
    lib.hif_solve.restype = i
    lib.hif_query_stats.argtypes = [vp, ctypes.POINTER(Stats)]
    lib.hif_query_stats.restype = i
    lib.hif_predict_bytes.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(Options)]
    lib.hif_predict_bytes.restype = ctypes.c_size_t
    lib.hif_profile_begin.argtypes = []
    lib.hif_profile_begin.restype = i
    lib.hif_profile_end.argtypes = [ctypes.POINTER(KernelProfile), i, ctypes.POINTER(ctypes.c_int)]
    lib.hif_profile_end.restype = i
    lib.hif_destroy.argtypes = [vp]
    lib.hif_destroy.restype = None
    lib.hif_save.argtypes = [vp, ctypes.c_char_p]
    lib.hif_save.restype = i
    lib.hif_load.argtypes = [ctypes.c_char_p, ctypes.POINTER(vp)]
    lib.hif_load.restype = i
    lib.hif_last_error.argtypes = []
    lib.hif_last_error.restype = ctypes.c_char_p
    lib.hif_version.argtypes = []
    lib.hif_version.restype = ctypes.c_char_p
    lib.hif_autotune.argtypes = [ctypes.POINTER(Grid), vp, vp, d, ctypes.POINTER(Options),
                                 ctypes.c_char_p, i, vp]
    lib.hif_autotune.restype = i
    lib.hif_autotune_load.argtypes = [ctypes.c_char_p]
    lib.hif_autotune_load.restype = i
    lib.hif_autotune_clear.argtypes = []
    lib.hif_autotune_clear.restype = None
    lib.hif_autotune_table.argtypes = [ctypes.c_char_p, ctypes.c_size_t,
                                       ctypes.POINTER(ctypes.c_size_t)]
    lib.hif_autotune_table.restype = i
    ptrs = ctypes.POINTER(vp)
    lib.hif_apply_batch.argtypes = [ptrs, i, ptrs, ptrs, ctypes.POINTER(ctypes.c_int), vp]
    lib.hif_apply_batch.restype = i
    lib.hif_solve_batch.argtypes = [ptrs, i, ptrs, ptrs, ctypes.POINTER(ctypes.c_int), vp,
                                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
    lib.hif_solve_batch.restype = i
    lib.hif_query_active.argtypes = [vp, i, ctypes.POINTER(ctypes.c_int32), ctypes.c_int64,
                                     ctypes.POINTER(ctypes.c_int64)]
    lib.hif_query_active.restype = i
    lib.hif_measure_peaks.argtypes = [ctypes.POINTER(Peaks), vp]
    lib.hif_measure_peaks.restype = i
    _lib = lib
    return lib


def _check(st: int):
    if st != HIF_OK:
        raise HifError(st, load().hif_last_error().decode())


def _ptr(x):
    """(pointer, keep-alive) for a torch tensor or numpy array of float64."""
    if x is None:
        return None, None
    try:
        import torch
        if isinstance(x, torch.Tensor):
            if x.dtype != torch.float64 or not x.is_contiguous():
                raise TypeError("tensors must be contiguous float64")
            return ctypes.c_void_p(x.data_ptr()), x
    except ImportError:  # pragma: no cover
        pass
    a = np.ascontiguousarray(x, dtype=np.float64)
    return ctypes.c_void_p(a.ctypes.data), a


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:  # pragma: no cover
            pass
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def default_options(**kw) -> Options:
    o = Options()
    load().hif_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def profile_begin():
    """Start timing every kernel the library launches (CUDA events)."""
    _check(load().hif_profile_begin())


def profile_end() -> list:
    """Stop timing; per-kernel dicts (name, launches, seconds, flops, bytes)."""
    cap = 128
    arr = (KernelProfile * cap)()
    cnt = ctypes.c_int()
    _check(load().hif_profile_end(arr, cap, ctypes.byref(cnt)))
    return [dict(name=arr[i].name.decode(), launches=arr[i].launches, kernels=arr[i].kernels,
                 seconds=arr[i].seconds, flops=arr[i].flops, bytes=arr[i].bytes)
            for i in range(min(cnt.value, cap))]


def measure_peaks(stream=None) -> dict:
    """hif_measure_peaks: measured FP32/FP64 FMA and TF32/BF16 tensor-core rates."""
    p = Peaks()
    _check(load().hif_measure_peaks(ctypes.byref(p), _stream(stream)))
    return {k: getattr(p, k) for k, _ in Peaks._fields_}


def predict_bytes(n: int, m: int, **opts) -> int:
    g = Grid(n, m, 0)
    o = default_options(**opts)
    return int(load().hif_predict_bytes(ctypes.byref(g), ctypes.byref(o)))


class Handle:
    """A factorization F ~= A held on the device (hif_factor / hif_destroy)."""

    def __init__(self, ptr: ctypes.c_void_p, n: int):
        self._h = ptr
        self.n = n
        self.N = n ** 3

    def close(self):
        if self._h:
            load().hif_destroy(self._h)
            self._h = None

    def save(self, path: str):
        """hif_save: write the factor to a file (hif_load reads it back)."""
        _check(load().hif_save(self._h, os.fsencode(path)))

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _nrhs(self, f):
        size = int(np.prod(tuple(f.shape)))
        if size % self.N:
            raise ValueError("right-hand side size is not a multiple of n^3")
        return size // self.N

    def apply(self, f, u, stream=None):
        """u = F^{-1} f (u preallocated, same shape and kind of memory as wanted)."""
        fp, _k1 = _ptr(f)
        up, _k2 = _ptr(u)
        _check(load().hif_apply(self._h, fp, up, self._nrhs(f), _stream(stream)))
        return u

    def apply_noalloc(self, f, u, stream=None):
        """u = F^{-1} f without any device allocation (f, u on the device).

        For callers that must not allocate device memory; the work space is the
        library's fixed 32 MiB device array (see hif_apply_noalloc in hif.h).
        """
        fp, _k1 = _ptr(f)
        up, _k2 = _ptr(u)
        _check(load().hif_apply_noalloc(self._h, fp, up, self._nrhs(f), _stream(stream)))
        return u

    def residual(self, f, u, r, stream=None):
        fp, _a = _ptr(f)
        up, _b = _ptr(u)
        rp, _c = _ptr(r)
        _check(load().hif_residual(self._h, fp, up, rp, self._nrhs(f), _stream(stream)))
        return r

    def solve(self, f, u, stream=None, check=True):
        """PCG solve of A u = f; returns (iterations, relative residuals) per column."""
        nrhs = self._nrhs(f)
        fp, _a = _ptr(f)
        up, _b = _ptr(u)
        its = (ctypes.c_int * nrhs)()
        rel = (ctypes.c_double * nrhs)()
        st = load().hif_solve(self._h, fp, up, nrhs, _stream(stream), its, rel)
        if check:
            _check(st)
        return list(its), list(rel)

    def active(self, level: int) -> np.ndarray:
        """hif_query_active: sorted grid indices active after `level`."""
        cnt = ctypes.c_int64()
        _check(load().hif_query_active(self._h, level, None, 0, ctypes.byref(cnt)))
        out = np.empty(cnt.value, dtype=np.int32)
        _check(load().hif_query_active(self._h, level,
                                       out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                       cnt.value, ctypes.byref(cnt)))
        return out

    def stats(self) -> dict:
        s = Stats()
        _check(load().hif_query_stats(self._h, ctypes.byref(s)))
        L = s.levels
        return dict(n=s.n, m=s.m, levels=L, precision=s.precision, eps=s.eps,
                    root_size=s.root_size, active_after=list(s.active_after)[:L],
                    fronts=[list(s.fronts[i]) for i in range(L + 1)],
                    factor_seconds=s.factor_seconds,
                    level_seconds=list(s.level_seconds)[:L + 1], flops=s.flops,
                    factor_bytes=s.factor_bytes, peak_bytes=s.peak_bytes,
                    stored_entries=s.stored_entries, kernel_launches=s.kernel_launches,
                    apply_launches=s.apply_launches, retried_fronts=s.retried_fronts)


def _batch_args(handles, fs, us):
    nh = len(handles)
    if not (nh == len(fs) == len(us)) or nh == 0:
        raise ValueError("need as many right-hand sides and outputs as handles")
    hp = (ctypes.c_void_p * nh)(*[h._h for h in handles])
    keep = []
    fp = (ctypes.c_void_p * nh)()
    up = (ctypes.c_void_p * nh)()
    nr = (ctypes.c_int * nh)()
    for k, (h, f, u) in enumerate(zip(handles, fs, us)):
        a, ka = _ptr(f)
        b, kb = _ptr(u)
        keep += [ka, kb]
        fp[k], up[k] = a.value, b.value
        nr[k] = h._nrhs(f)
    return hp, fp, up, nr, keep


def apply_batch(handles, fs, us, stream=None):
    """hif_apply_batch: us[i] = F_i^{-1} fs[i] with the sweeps of every factor in
    shared launches (bitwise each handle's own apply)."""
    hp, fp, up, nr, _keep = _batch_args(handles, fs, us)
    _check(load().hif_apply_batch(hp, len(handles), fp, up, nr, _stream(stream)))
    return us


def solve_batch(handles, fs, us, stream=None, check=True):
    """hif_solve_batch: PCG of every system in lockstep, preconditioner applied
    as one grouped apply; returns per system (iterations, relative residuals)."""
    hp, fp, up, nr, _keep = _batch_args(handles, fs, us)
    tot = sum(nr)
    its = (ctypes.c_int * tot)()
    rel = (ctypes.c_double * tot)()
    st = load().hif_solve_batch(hp, len(handles), fp, up, nr, _stream(stream), its, rel)
    if check:
        _check(st)
    out, c = [], 0
    for k in range(len(handles)):
        out.append((list(its[c:c + nr[k]]), list(rel[c:c + nr[k]])))
        c += nr[k]
    return out


def autotune(n: int, m: int, a, b=None, b_const: float = 0.0, eps: float = 1e-6,
             precision: int = PREC_FP32, path: str | None = None, force: bool = False,
             stream=None, periodic: bool = False, **opts) -> str:
    """hif_autotune on this operator; returns the table (text) now in use."""
    g = Grid(n, m, 1 if periodic else 0)
    o = default_options(eps=eps, precision=precision, **opts)
    ap, _ka = _ptr(a)
    bp, _kb = _ptr(b)
    _check(load().hif_autotune(ctypes.byref(g), ap, bp, float(b_const), ctypes.byref(o),
                               os.fsencode(path) if path else None, int(bool(force)),
                               _stream(stream)))
    return autotune_table()


def autotune_load(path: str):
    _check(load().hif_autotune_load(os.fsencode(path)))


def autotune_clear():
    load().hif_autotune_clear()


def autotune_table() -> str:
    n = ctypes.c_size_t()
    _check(load().hif_autotune_table(None, 0, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value + 1)
    _check(load().hif_autotune_table(buf, n.value + 1, ctypes.byref(n)))
    return buf.value.decode()


def load_factor(path: str) -> Handle:
    """hif_load: a handle from a file written by Handle.save."""
    out = ctypes.c_void_p()
    _check(load().hif_load(os.fsencode(path), ctypes.byref(out)))
    s = Stats()
    _check(load().hif_query_stats(out, ctypes.byref(s)))
    return Handle(out, s.n)


def factor(n: int, m: int, a, b=None, b_const: float = 0.0, eps: float = 1e-6,
           precision: int = PREC_FP64, pcg_tol: float = 1e-10, max_iter: int = 200,
           stream=None, tensor_cores: bool = True, use_graphs: bool = True,
           retry_growth: float | None = None, periodic: bool = False) -> Handle:
    """hif_factor: a (and b) are n^3 float64 arrays, host or device.
    periodic=True: the periodic grid (hif_grid.bc = 1), b > 0 required."""
    g = Grid(n, m, 1 if periodic else 0)
    o = default_options(eps=eps, precision=precision, pcg_tol=pcg_tol, max_iter=max_iter,
                        tensor_cores=int(bool(tensor_cores)), use_graphs=int(bool(use_graphs)))
    if retry_growth is not None:
        o.retry_growth = float(retry_growth)
    ap, _ka = _ptr(a)
    bp, _kb = _ptr(b)
    out = ctypes.c_void_p()
    _check(load().hif_factor(ctypes.byref(g), ap, bp, float(b_const), ctypes.byref(o),
                             _stream(stream), ctypes.byref(out)))
    return Handle(out, n)
