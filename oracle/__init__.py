"""CPU oracle for C = A.B: the checker of the CUDA path.

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path (package ``paper_1306_6192_gb300``) and neither imports the
other; both take their inputs from ``synth``.

What it computes is the plain definition of the Cauchy product (paper, Section
"Implementacje algorytmow": c_ij = sum_r a_ir b_rj) in the order of the
sequential algorithm of Listing 1, in FP64, plus accurate entry checks (Dot2,
long double, exact fixed point for powers of two).  See oracle.c.

Error metric (the paper gives none; the reading used throughout):
    e_ij = |c_hat_ij - c_ij| / (|A|.|B|)_ij
with (|A|.|B|)_ij = sum_r |a_ir| |b_rj|; where that normaliser is 0 the entry
must be exactly 0 (e_ij = inf otherwise).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None
_i64 = ctypes.c_int64
_dp = ctypes.POINTER(ctypes.c_double)
_lp = ctypes.POINTER(ctypes.c_int64)


def _bind(lib):
    lib.oracle_gemm_f64.argtypes = [_i64, _i64, _i64, _dp, _dp, _dp, _dp, ctypes.c_int]
    lib.oracle_gemm_f64.restype = ctypes.c_int
    lib.oracle_entries_dot2.argtypes = [_i64, _i64, _i64, _dp, _dp, _i64, _lp, _lp, _dp, _dp, _dp]
    lib.oracle_entries_dot2.restype = None
    lib.oracle_entries_ld.argtypes = [_i64, _i64, _i64, _dp, _dp, _i64, _lp, _lp, _dp, _dp]
    lib.oracle_entries_ld.restype = None
    lib.oracle_gemv_dot2.argtypes = [_i64, _i64, _dp, _dp, _dp, _dp]
    lib.oracle_gemv_dot2.restype = None
    lib.oracle_gemm_pow2_exact.argtypes = [_i64, _i64, _i64, _dp, _dp, ctypes.c_int, _dp, _dp]
    lib.oracle_gemm_pow2_exact.restype = _i64
    lib.oracle_cgemm_f64.argtypes = [_i64, _i64, _i64, _dp, _dp, _dp, _dp]
    lib.oracle_cgemm_f64.restype = None
    lib.oracle_default_threads.restype = ctypes.c_int
    lib.oracle_ldbl_mant_dig.restype = ctypes.c_int
    lib.oracle_mutant.restype = ctypes.c_int
    return lib


def load(path: str | None = None):
    """Loads the oracle library (building it first if needed).  With ``path``
    a specific build (e.g. a mutant) is loaded and returned as an Oracle."""
    global _lib
    if path is not None:
        return Oracle(_bind(ctypes.CDLL(path)))
    if _lib is None:
        _lib = _bind(ctypes.CDLL(_build.build()))
    return _lib


def _p(a):
    return a.ctypes.data_as(_dp)


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


class Oracle:
    """The oracle's entry points bound to one loaded library."""

    def __init__(self, lib=None):
        self.lib = lib if lib is not None else load()

    # -- plain definition in FP64 (Listing 1 order) -------------------------
    def gemm(self, A, B, threads: int = 0, with_abs: bool = False):
        A = _f64(A); B = _f64(B)
        n, m = A.shape
        m2, p = B.shape
        assert m == m2, "inner dimensions differ"
        C = np.empty((n, p), np.float64)
        absC = np.empty((n, p), np.float64) if with_abs else None
        rc = self.lib.oracle_gemm_f64(n, m, p, _p(A), _p(B), _p(C),
                                      _p(absC) if with_abs else None, threads)
        if rc != 0:
            raise MemoryError("oracle_gemm_f64 failed")
        return (C, absC) if with_abs else C

    # -- accurate entries ---------------------------------------------------
    def axpby(self, alpha, A, B, beta, D, threads: int = 0):
        """alpha (A.B) + beta D: the product with the matrix addition /
        subtraction of the paper's results section on top, in FP64, and the
        normaliser of its entry errors, |alpha| (|A|.|B|) + |beta| |D|.
        alpha == 0 leaves the product out (A and B are not used) and
        beta == 0 leaves D out (it may be None), as zero terms."""
        alpha, beta = float(alpha), float(beta)
        if alpha != 0.0:
            ref, ab = self.gemm(A, B, threads=threads, with_abs=True)
            out, norm = alpha * ref, abs(alpha) * ab
        else:
            shape = np.shape(D)  # C has D's shape
            out, norm = np.zeros(shape), np.zeros(shape)
        if beta != 0.0:
            d = np.asarray(D, np.float64)
            out = out + beta * d
            norm = norm + abs(beta) * np.abs(d)
        return out, norm

    def entries(self, A, B, I, J, method: str = "dot2"):
        """c_ij for the sampled (I, J) as (hi, lo, |A||B|_ij)."""
        A = _f64(A); B = _f64(B)
        n, m = A.shape
        p = B.shape[1]
        I = np.ascontiguousarray(I, np.int64); J = np.ascontiguousarray(J, np.int64)
        c = len(I)
        hi = np.empty(c); lo = np.empty(c); ab = np.empty(c)
        if method == "dot2":
            self.lib.oracle_entries_dot2(n, m, p, _p(A), _p(B), c,
                                         I.ctypes.data_as(_lp), J.ctypes.data_as(_lp),
                                         _p(hi), _p(lo), _p(ab))
        elif method == "ld":
            self.lib.oracle_entries_dot2(n, m, p, _p(A), _p(B), c,
                                         I.ctypes.data_as(_lp), J.ctypes.data_as(_lp),
                                         _p(np.empty(c)), _p(np.empty(c)), _p(ab))
            self.lib.oracle_entries_ld(n, m, p, _p(A), _p(B), c,
                                       I.ctypes.data_as(_lp), J.ctypes.data_as(_lp),
                                       _p(hi), _p(lo))
        else:
            raise ValueError(method)
        return hi, lo, ab

    def gemv(self, X, v):
        """y = X.v (Dot2 per row) and |X|.|v|."""
        X = _f64(X); v = _f64(v)
        r, c = X.shape
        y = np.empty(r); ya = np.empty(r)
        self.lib.oracle_gemv_dot2(r, c, _p(X), _p(v), _p(y), _p(ya))
        return y, ya

    def freivalds_rhs(self, A, B, x):
        """z = A.(B.x) and its normaliser |A|.(|B|.|x|), both via Dot2 gemv."""
        w, _ = self.gemv(B, x)
        z, _ = self.gemv(A, w)
        wa, _ = self.gemv(np.abs(_f64(B)), np.abs(_f64(x)))
        za, _ = self.gemv(np.abs(_f64(A)), wa)
        return z, za

    def cgemm(self, A, B):
        """Complex C = A.B in FP64 (Listing 1 order) and |A|.|B| (moduli)."""
        A = np.ascontiguousarray(A, np.complex128)
        B = np.ascontiguousarray(B, np.complex128)
        n, m = A.shape
        p = B.shape[1]
        C = np.empty((n, p), np.complex128)
        absC = np.empty((n, p), np.float64)
        self.lib.oracle_cgemm_f64(n, m, p, A.ctypes.data_as(_dp), B.ctypes.data_as(_dp),
                                  C.ctypes.data_as(_dp), _p(absC))
        return C, absC

    def pow2_exact(self, A, B, shift: int = 50):
        """Exact C for inputs that are 0 or +-2^k: (hi, lo) doubles."""
        A = _f64(A); B = _f64(B)
        n, m = A.shape
        p = B.shape[1]
        hi = np.empty((n, p)); lo = np.empty((n, p))
        rc = self.lib.oracle_gemm_pow2_exact(n, m, p, _p(A), _p(B), shift, _p(hi), _p(lo))
        if rc != 0:
            raise ValueError("pow2_exact: input entry %d outside the exact range" % (-rc - 1))
        return hi, lo

    def default_threads(self) -> int:
        return int(self.lib.oracle_default_threads())

    def ldbl_mant_dig(self) -> int:
        return int(self.lib.oracle_ldbl_mant_dig())

    def mutant(self) -> int:
        return int(self.lib.oracle_mutant())


_default = None


def default() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle()
    return _default


# -- error metric ---------------------------------------------------------------

def rel_errors(c_hat, c_ref, abs_ref):
    """e = |c_hat - c_ref| / abs_ref elementwise; where abs_ref == 0 the entry
    must be exact: 0 if c_hat == c_ref (signed zeros compare equal), inf
    otherwise.  A NaN on either side, or infinities that do not cancel to a
    finite difference, give inf: a non-finite entry is never within a
    tolerance (tests of NaN/inf propagation check those entries directly)."""
    c_hat = np.asarray(c_hat, np.float64)
    c_ref = np.asarray(c_ref, np.float64)
    abs_ref = np.asarray(abs_ref, np.float64)
    with np.errstate(invalid="ignore"):
        diff = np.abs(c_hat - c_ref)
    with np.errstate(divide="ignore", invalid="ignore"):
        e = np.where(abs_ref > 0, diff / np.where(abs_ref > 0, abs_ref, 1.0),
                     np.where(diff == 0, 0.0, np.inf))
    return np.where(np.isnan(diff), np.inf, e)


def rel_errors_complex(c_hat, c_ref, abs_ref):
    """Complex version of rel_errors: |c_hat - c_ref| (modulus) / abs_ref."""
    c_hat = np.asarray(c_hat, np.complex128)
    c_ref = np.asarray(c_ref, np.complex128)
    abs_ref = np.asarray(abs_ref, np.float64)
    diff = np.abs(c_hat - c_ref)
    with np.errstate(divide="ignore", invalid="ignore"):
        e = np.where(abs_ref > 0, diff / np.where(abs_ref > 0, abs_ref, 1.0),
                     np.where(diff == 0, 0.0, np.inf))
    return np.where(np.isnan(diff), np.inf, e)


def tolerance(m: int, dtype: str) -> float:
    """Stated tolerance on max e_ij: 1e-6*sqrt(m) for the FP32-accuracy paths,
    1e-14*sqrt(m) for FP64 (m = inner dimension, at least 1)."""
    m = max(int(m), 1)
    if dtype in ("f32", "simt", "split"):
        return 1e-6 * np.sqrt(m)
    if dtype in ("f64", "dgemm"):
        return 1e-14 * np.sqrt(m)
    if dtype == "c32":
        # each part of a complex entry is a difference/sum of two real
        # products, each within 1e-6 sqrt(m) of its own normaliser <= |A||B|
        return 2e-6 * np.sqrt(m)
    raise ValueError(dtype)


def normwise_error(c_hat, c_ref) -> float:
    """max |c_hat - c_ref| / max |c_ref| over all entries (reported, never a
    gate); the plain max difference when c_ref is all zero, 0 when empty."""
    c_ref = np.asarray(c_ref, np.float64)
    mx = float(np.max(np.abs(c_ref))) if c_ref.size else 0.0
    d = float(np.max(np.abs(np.asarray(c_hat, np.float64) - c_ref))) if c_ref.size else 0.0
    return d / mx if mx > 0 else d
