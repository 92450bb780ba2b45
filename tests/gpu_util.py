"""Helpers of the GPU parity tests: device copies, oracle comparisons."""
from __future__ import annotations

import numpy as np
import torch

import oracle
import synth

F32_TOL = "f32"
F64_TOL = "f64"


def dev(x, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def run_gemm(mm, A, B, mode, f64=False, out_fill=float("nan")):
    """C = A.B through mm_gemm on device copies; returns the numpy result."""
    n, m = A.shape
    p = B.shape[1]
    dt = mm.MM_F64 if f64 else mm.MM_F32
    tdt = torch.float64 if f64 else torch.float32
    dA = dev(A, tdt)
    dB = dev(B, tdt)
    dC = torch.full((n, p), out_fill, dtype=tdt, device="cuda")
    st = mm.mm_gemm(n, m, p, dA, dB, dC, dt, mode)
    assert st == mm.MM_OK, mm.mm_strerror(st)
    return dC.cpu().numpy()


def run_packed(mm, A, B, mode):
    """C = A.B as a grouped call of this one product: the packed split path
    (pack, verify, fix, persistent tcgen05 kernel with its tail split), which
    grouped calls and serving batches use for every product.  mm_gemm runs
    products with few output tiles on the fused split-K kernel instead."""
    n, m = A.shape
    p = B.shape[1]
    dA, dB = dev(A), dev(B)
    dC = torch.full((n, p), float("nan"), device="cuda")
    st = mm.mm_gemm_grouped([(n, m, p, dA, dB, dC)], mm.MM_F32, mode)
    assert st == mm.MM_OK, mm.mm_strerror(st)
    return dC.cpu().numpy()


def fused_slices(mm, n, m, p):
    """Slices of the fused split-K plan of an n x m x p split product (0: the
    product takes the packed path)."""
    st, _, slices, _, _ = mm.mm_tune_query_splitk(n, m, p)
    assert st == mm.MM_OK
    return slices


def full_errors(C, A, B, orc=None):
    orc = orc or oracle.default()
    ref, absref = orc.gemm(A, B, with_abs=True)
    return oracle.rel_errors(C, ref, absref), ref


def assert_full(C, A, B, kind):
    e, _ = full_errors(C, A, B)
    m = A.shape[1]
    tol = oracle.tolerance(m, kind)
    assert e.size == 0 or e.max() <= tol, "max e = %g > tol %g" % (e.max(), tol)
    return float(e.max()) if e.size else 0.0


def sampled_check(C, A, B, kind, seed=2, count=4096, trials=2, kappa=4.0):
    """4096 sampled entries against Dot2 and two Freivalds trials, both with
    the |A||B| normaliser; returns (max entry error, max Freivalds ratio)."""
    orc = oracle.default()
    n, m = A.shape
    p = B.shape[1]
    tol = oracle.tolerance(m, kind)
    I, J = synth.sample_indices(seed, n, p, count)
    hi, lo, ab = orc.entries(A, B, I, J, "dot2")
    e = oracle.rel_errors(C[I, J].astype(np.float64), hi + lo, ab)
    emax = float(e.max())
    assert emax <= tol, "sampled max e = %g > %g" % (emax, tol)
    fmax = 0.0
    for t in range(trials):
        x = synth.freivalds_vector(seed + 100 + t, p)
        y, _ = orc.gemv(C.astype(np.float64), x)
        z, za = orc.freivalds_rhs(A, B, x)
        r = np.abs(y - z) / np.where(za > 0, za, 1.0)
        fmax = max(fmax, float(r.max()))
    assert fmax <= kappa * tol, "Freivalds ratio %g > %g" % (fmax, kappa * tol)
    return emax, fmax
