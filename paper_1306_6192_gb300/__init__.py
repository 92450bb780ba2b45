"""Python binding of the mm C ABI (include/mm.h): argument marshalling only.

Every function has the C name and returns the C status code (an int, 0 on
success) plus any output values; ``check_status`` turns a code into an
exception.  Operands may be torch tensors (device or host), numpy arrays (host)
or raw integer addresses.  Every step of the product runs in the CUDA library
``libmm_gb300.so``; when it has not been built this module raises on first use
instead of falling back to anything else.
"""
from __future__ import annotations

import atexit
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmm_gb300.so")

# status codes
MM_OK, MM_EINVAL, MM_ENOMEM, MM_EBUDGET, MM_EBUSY, MM_ENOTFOUND = 0, 1, 2, 3, 4, 5
MM_EPENDING, MM_ETIMEOUT, MM_ECUDA, MM_ENOTINIT, MM_EUNSUPPORTED, MM_ECANCELLED = 6, 7, 8, 9, 10, 11
MM_ESCRATCH = 12
# element types and modes
MM_F32, MM_F64 = 0, 1
MM_MODE_SIMT, MM_MODE_SPLIT_BF16X3, MM_MODE_DGEMM, MM_MODE_FP8, MM_MODE_AUTO = 0, 1, 2, 3, 4
MM_MODE_OZAKI = 5
MM_MODE_SPLIT_BF16X6 = 6

_i64 = ctypes.c_int64
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)


class mm_opts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("n_streams", ctypes.c_int),
                ("tune_table", ctypes.c_char_p), ("check", ctypes.c_int),
                ("device", ctypes.c_int), ("max_batch", ctypes.c_int)]


class mm_problem(ctypes.Structure):
    _fields_ = [("n", _i64), ("m", _i64), ("p", _i64), ("A", _vp), ("B", _vp), ("C", _vp)]


class MMError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = status
        super().__init__("%s: %s (%d)" % (where or "mm", mm_strerror(status), status))


_lib = None


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                "libmm_gb300.so is missing: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        st = ctypes.c_int
        L.mm_strerror.argtypes = [st]
        L.mm_strerror.restype = ctypes.c_char_p
        L.mm_init.argtypes = [ctypes.POINTER(mm_opts)]
        L.mm_shutdown.argtypes = []
        L.mm_gemm.argtypes = [_i64, _i64, _i64, _vp, _vp, _vp, st, st]
        L.mm_gemm_async.argtypes = [_i64, _i64, _i64, _vp, _vp, _vp, st, st, _vp]
        _dbl = ctypes.c_double
        L.mm_gemm_axpby.argtypes = [_i64, _i64, _i64, _dbl, _vp, _vp, _dbl, _vp, _vp, st, st]
        L.mm_gemm_axpby_async.argtypes = [_i64, _i64, _i64, _dbl, _vp, _vp, _dbl, _vp, _vp, st, st,
                                          _vp]
        L.mm_gemm_grouped.argtypes = [ctypes.c_int32, ctypes.POINTER(mm_problem), st, st]
        L.mm_gemm_grouped_async.argtypes = [ctypes.c_int32, ctypes.POINTER(mm_problem), st, st,
                                            _vp]
        L.mm_sync.argtypes = [_vp]
        L.mm_check.argtypes = [_i64, _i64, _i64, _vp, _vp, _vp, st, _vp, _i64, _vp, _vp, _dp]
        L.mm_submit.argtypes = [ctypes.POINTER(mm_problem), st, st, ctypes.POINTER(ctypes.c_uint64)]
        L.mm_poll.argtypes = [ctypes.c_uint64, ctypes.POINTER(ctypes.c_int), _dp, _dp]
        L.mm_wait.argtypes = [ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(ctypes.c_int), _dp,
                              _dp]
        L.mm_serve_stats.argtypes = [ctypes.POINTER(_i64)] * 4
        L.mm_tune.argtypes = [_i64, _i64, _i64, ctypes.c_int]
        L.mm_tune_save.argtypes = [ctypes.c_char_p]
        L.mm_tune_load.argtypes = [ctypes.c_char_p]
        L.mm_tune_query.argtypes = [_i64, _i64, _i64] + [ctypes.POINTER(ctypes.c_int)] * 4
        L.mm_tune_query_tail.argtypes = [_i64, _i64, _i64] + [ctypes.POINTER(ctypes.c_int)] * 3
        L.mm_tune_query_splitk.argtypes = [_i64, _i64, _i64] + [ctypes.POINTER(ctypes.c_int)] * 4
        L.mm_tail_plan.argtypes = [_i64, ctypes.c_int, ctypes.c_int, ctypes.c_int, _i64,
                                   ctypes.c_double] + [ctypes.POINTER(ctypes.c_int)] * 2
        L.mm_simt_plan.argtypes = [_i64, _i64, _i64, ctypes.c_int, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_i64),
                                   ctypes.POINTER(ctypes.c_int)]
        L.mm_trace_enable.argtypes = [ctypes.c_int]
        L.mm_trace_reset.argtypes = []
        L.mm_trace_read.argtypes = [ctypes.c_char_p, ctypes.POINTER(_i64), _dp]
        L.mm_launch_count.argtypes = []
        L.mm_launch_count.restype = _i64
        L.mm_cgemm.argtypes = [_i64, _i64, _i64, _vp, _vp, _vp, st]
        L.mm_add.argtypes = [_i64, _i64, ctypes.c_double, _vp, ctypes.c_double, _vp, _vp, st]
        L.mm_diag.argtypes = [_i64, _i64, _vp, _vp, _vp, ctypes.c_int, st]
        L.mm_add_async.argtypes = [_i64, _i64, ctypes.c_double, _vp, ctypes.c_double, _vp, _vp, st,
                                   _vp]
        L.mm_diag_async.argtypes = [_i64, _i64, _vp, _vp, _vp, ctypes.c_int, st, _vp]
        for name in ("mm_cgemm", "mm_add", "mm_diag", "mm_add_async", "mm_diag_async"):
            getattr(L, name).restype = ctypes.c_int
        L.mm_gemm_split_static.argtypes = [_i64, _i64, _i64, _vp, _vp, _vp, _vp]
        L.mm_gemm_split_static.restype = ctypes.c_int
        L.mm_measure_fma_peak.argtypes = [st, _i64, _dp]
        L.mm_measure_fma_peak.restype = ctypes.c_int
        L.mm_ozaki_slices.argtypes = [ctypes.c_int]
        L.mm_ozaki_gate.argtypes = [ctypes.c_int]
        L.mm_ozaki_gate.restype = ctypes.c_int
        L.mm_ozaki_slices.restype = ctypes.c_int
        L.mm_ozaki_plan.argtypes = [_i64, _i64, _i64, ctypes.c_int, ctypes.POINTER(_i64),
                                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_size_t)]
        L.mm_ozaki_plan.restype = ctypes.c_int
        for name in ("mm_init", "mm_shutdown", "mm_gemm", "mm_gemm_async", "mm_gemm_axpby",
                     "mm_gemm_axpby_async", "mm_gemm_grouped",
                     "mm_gemm_grouped_async", "mm_sync", "mm_check", "mm_submit", "mm_poll",
                     "mm_wait", "mm_serve_stats", "mm_tune", "mm_tune_save", "mm_tune_load",
                     "mm_tune_query", "mm_tune_query_tail", "mm_tune_query_splitk",
                     "mm_tail_plan", "mm_simt_plan", "mm_trace_enable",
                     "mm_trace_reset", "mm_trace_read"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
        atexit.register(_shutdown_at_exit)
    return _lib


def _shutdown_at_exit():
    # stops the serving thread and frees library memory while CUDA is alive
    if _lib is not None:
        _lib.mm_shutdown()


def _ptr(x):
    """Address of a torch tensor / numpy array / int (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError("cannot take the address of %r" % type(x))


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream  # torch.cuda.Stream / ExternalStream


def check_status(st: int, where: str = "") -> None:
    if st != MM_OK:
        raise MMError(st, where)


def mm_strerror(st: int) -> str:
    return lib().mm_strerror(int(st)).decode()


# Tuning table measured on GB300 (tune_gb300.py); loaded unless another is given.
DEFAULT_TUNE_TABLE = os.path.join(HERE, "tune_gb300.txt")


def mm_init(hbm_budget_bytes: int = 0, n_streams: int = 0, tune_table: str | None = None,
            check: int = 0, device: int = -1, max_batch: int = 0) -> int:
    if tune_table is None and os.path.exists(DEFAULT_TUNE_TABLE):
        tune_table = DEFAULT_TUNE_TABLE
    o = mm_opts(hbm_budget_bytes, n_streams, tune_table.encode() if tune_table else None,
                check, device, max_batch)
    return lib().mm_init(ctypes.byref(o))


def mm_shutdown() -> int:
    return lib().mm_shutdown()


def mm_gemm(n, m, p, A, B, C, dt, mode) -> int:
    return lib().mm_gemm(n, m, p, _ptr(A), _ptr(B), _ptr(C), dt, mode)


def mm_gemm_async(n, m, p, A, B, C, dt, mode, stream=None) -> int:
    return lib().mm_gemm_async(n, m, p, _ptr(A), _ptr(B), _ptr(C), dt, mode, _stream(stream))


def mm_gemm_axpby(n, m, p, alpha, A, B, beta, D, C, dt, mode) -> int:
    """C = alpha (A.B) + beta D with the epilogue fused into the product
    (device matrices; D may be C itself or None where beta == 0)."""
    return lib().mm_gemm_axpby(n, m, p, float(alpha), _ptr(A), _ptr(B), float(beta), _ptr(D),
                               _ptr(C), dt, mode)


def mm_gemm_axpby_async(n, m, p, alpha, A, B, beta, D, C, dt, mode, stream=None) -> int:
    return lib().mm_gemm_axpby_async(n, m, p, float(alpha), _ptr(A), _ptr(B), float(beta),
                                     _ptr(D), _ptr(C), dt, mode, _stream(stream))


def mm_problems(probs):
    """A ctypes array of mm_problem from (n, m, p, A, B, C) tuples; pass it
    to the grouped calls to marshal a large table only once."""
    if isinstance(probs, ctypes.Array):
        return probs
    arr = (mm_problem * max(len(probs), 1))()
    for k, (n, m, p, A, B, C) in enumerate(probs):
        arr[k] = mm_problem(n, m, p, _ptr(A), _ptr(B), _ptr(C))
    return arr


def mm_gemm_grouped(probs, dt, mode) -> int:
    """probs: sequence of (n, m, p, A, B, C)."""
    return lib().mm_gemm_grouped(len(probs), mm_problems(probs), dt, mode)


def mm_gemm_grouped_async(probs, dt, mode, stream=None) -> int:
    return lib().mm_gemm_grouped_async(len(probs), mm_problems(probs), dt, mode, _stream(stream))


def mm_sync(stream=None) -> int:
    return lib().mm_sync(_stream(stream))


def mm_check(n, m, p, A, B, C, dt, x, I=None, J=None):
    """Returns (status, freivalds_max_residual, sampled_max_error)."""
    out = (ctypes.c_double * 2)()
    ns = 0 if I is None else int(I.numel() if hasattr(I, "numel") else len(I))
    st = lib().mm_check(n, m, p, _ptr(A), _ptr(B), _ptr(C), dt, _ptr(x), ns, _ptr(I), _ptr(J),
                        out)
    return st, out[0], out[1]


def mm_submit(n, m, p, A, B, C, dt, mode):
    """Returns (status, request id)."""
    q = mm_problem(n, m, p, _ptr(A), _ptr(B), _ptr(C))
    rid = ctypes.c_uint64(0)
    st = lib().mm_submit(ctypes.byref(q), dt, mode, ctypes.byref(rid))
    return st, rid.value


def mm_poll(rid):
    """Returns (status, result status, checked error, latency ms)."""
    r = ctypes.c_int(0)
    e = ctypes.c_double(0)
    t = ctypes.c_double(0)
    st = lib().mm_poll(rid, ctypes.byref(r), ctypes.byref(e), ctypes.byref(t))
    return st, r.value, e.value, t.value


def mm_wait(rid, timeout_s: float = 60.0):
    r = ctypes.c_int(0)
    e = ctypes.c_double(0)
    t = ctypes.c_double(0)
    st = lib().mm_wait(rid, timeout_s, ctypes.byref(r), ctypes.byref(e), ctypes.byref(t))
    return st, r.value, e.value, t.value


def mm_serve_stats():
    v = [_i64(0) for _ in range(4)]
    st = lib().mm_serve_stats(*[ctypes.byref(x) for x in v])
    return (st,) + tuple(x.value for x in v)


def mm_tune(n, m, p, reps: int = 3) -> int:
    return lib().mm_tune(n, m, p, reps)


def mm_tune_save(path: str) -> int:
    return lib().mm_tune_save(path.encode())


def mm_tune_load(path: str) -> int:
    return lib().mm_tune_load(path.encode())


def mm_tune_query(n, m, p):
    """Returns (status, bn, bk, stages, group_m)."""
    v = [ctypes.c_int(0) for _ in range(4)]
    st = lib().mm_tune_query(n, m, p, *[ctypes.byref(x) for x in v])
    return (st,) + tuple(x.value for x in v)


def mm_tune_query_tail(n, m, p):
    """Returns (status, tiles, split_from, split_s) of the split path's tail
    split for one n x m x p product."""
    v = [ctypes.c_int(0) for _ in range(3)]
    st = lib().mm_tune_query_tail(n, m, p, *[ctypes.byref(x) for x in v])
    return (st,) + tuple(x.value for x in v)


def mm_tune_query_splitk(n, m, p):
    """Returns (status, tiles, slices, clusters, cluster_size) of the fused
    split-K plan of one n x m x p split product (slices = 0: packed path)."""
    v = [ctypes.c_int(0) for _ in range(4)]
    st = lib().mm_tune_query_splitk(n, m, p, *[ctypes.byref(x) for x in v])
    return (st,) + tuple(x.value for x in v)


def mm_simt_plan(n, m, p, dt, sms: int = 0):
    """Returns (status, slices, slice_k, tile) of the K-slice plan of a SIMT
    (MM_F32) or DGEMM (MM_F64) product (slices = 0: the one-pass kernel).
    Needs no device."""
    s, k, t = ctypes.c_int(0), _i64(0), ctypes.c_int(0)
    st = lib().mm_simt_plan(n, m, p, dt, sms, ctypes.byref(s), ctypes.byref(k), ctypes.byref(t))
    return st, s.value, k.value, t.value


def mm_measure_fma_peak(dt, iters: int = 4096):
    """Returns (status, flops per second) of the CUDA cores' FMA for dt."""
    v = ctypes.c_double(0.0)
    st = lib().mm_measure_fma_peak(dt, iters, ctypes.byref(v))
    return st, v.value


def mm_tail_plan(tiles, grid, kt, bn, m, products):
    """Returns (status, split_from, split_s) of the tail-split planner (a
    pure host function; no GPU needed)."""
    a, b = ctypes.c_int(0), ctypes.c_int(0)
    st = lib().mm_tail_plan(tiles, grid, kt, bn, m, float(products), ctypes.byref(a),
                            ctypes.byref(b))
    return st, a.value, b.value


def mm_ozaki_slices(slices: int) -> int:
    """Digit slices S (2..12) of MM_MODE_OZAKI for the products queued next."""
    return lib().mm_ozaki_slices(int(slices))


def mm_ozaki_gate(on: int) -> int:
    """Turns the accuracy gate of MM_MODE_OZAKI products on (1) or off (0)."""
    return lib().mm_ozaki_gate(on)


def mm_ozaki_plan(n, m, p, slices):
    """Returns (status, K columns per chunk, chunks, scratch bytes bound) of an
    MM_MODE_OZAKI product (a pure host function; no GPU needed)."""
    mc, q, b = _i64(0), ctypes.c_int(0), ctypes.c_size_t(0)
    st = lib().mm_ozaki_plan(n, m, p, int(slices), ctypes.byref(mc), ctypes.byref(q),
                             ctypes.byref(b))
    return st, mc.value, q.value, b.value


def mm_trace_enable(on: bool = True) -> int:
    return lib().mm_trace_enable(1 if on else 0)


def mm_trace_reset() -> int:
    return lib().mm_trace_reset()


def mm_trace_read(kernel: str):
    """Returns (status, launches, total device ms) of one kernel name."""
    n = _i64(0)
    ms = ctypes.c_double(0)
    st = lib().mm_trace_read(kernel.encode(), ctypes.byref(n), ctypes.byref(ms))
    return st, n.value, ms.value


def mm_launch_count() -> int:
    return int(lib().mm_launch_count())


def mm_cgemm(n, m, p, A, B, C, mode) -> int:
    """Complex product of complex64 device matrices (see include/mm.h)."""
    return lib().mm_cgemm(n, m, p, _ptr(A), _ptr(B), _ptr(C), mode)


def mm_add(n, p, alpha, A, beta, B, C, dt) -> int:
    """C = alpha A + beta B elementwise (device matrices)."""
    return lib().mm_add(n, p, float(alpha), _ptr(A), float(beta), _ptr(B), _ptr(C), dt)


def mm_diag(n, p, X, d, C, side, dt) -> int:
    """side 0: C = X.diag(d); side 1: C = diag(d).X (device matrices)."""
    return lib().mm_diag(n, p, _ptr(X), _ptr(d), _ptr(C), side, dt)


def mm_add_async(n, p, alpha, A, beta, B, C, dt, stream=None) -> int:
    return lib().mm_add_async(n, p, float(alpha), _ptr(A), float(beta), _ptr(B), _ptr(C), dt,
                              _stream(stream))


def mm_diag_async(n, p, X, d, C, side, dt, stream=None) -> int:
    return lib().mm_diag_async(n, p, _ptr(X), _ptr(d), _ptr(C), side, dt, _stream(stream))


def mm_gemm_split_static(n, m, p, A, B, C, stream=None) -> int:
    """Allocation-free split product (see include/mm.h): device operands,
    scratch in the library's fixed device array, synchronous on `stream`."""
    return lib().mm_gemm_split_static(n, m, p, _ptr(A), _ptr(B), _ptr(C), _stream(stream))
