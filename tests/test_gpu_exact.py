"""Exact pins on the GPU paths: integer inputs, identity, diagonal (the
paper's special case), powers of two, empty sizes, the transpose identity."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import assert_full, dev, run_gemm

pytestmark = pytest.mark.gpu

MODES = ["simt", "split", "dgemm"]


def _md(mm, mode):
    return {"simt": mm.MM_MODE_SIMT, "split": mm.MM_MODE_SPLIT_BF16X3,
            "dgemm": mm.MM_MODE_DGEMM}[mode]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("shape", [(64, 64, 64), (129, 4096, 70), (300, 517, 260)])
def test_small_integers_bit_exact(mmlib, mode, shape):
    """Entries in [-8, 8]: |c| <= 64 m < 2^24, every partial sum is an exact
    integer in FP32 (and bf16 holds such integers exactly, lo = 0), so every
    path must reproduce the exact integer product bit for bit."""
    n, m, p = shape
    A = synth.small_ints(51, (n, m))
    B = synth.small_ints(52, (m, p))
    C = run_gemm(mmlib, A, B, _md(mmlib, mode), f64=(mode == "dgemm"))
    exact = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
    assert np.array_equal(C.astype(np.float64), exact)


@pytest.mark.parametrize("mode", MODES)
def test_identity(mmlib, mode):
    A = synth.uniform_pm1(61, (150, 140))
    C = run_gemm(mmlib, A, synth.identity(140), _md(mmlib, mode), f64=(mode == "dgemm"))
    if mode == "split":
        # hi + lo keeps 16 of the 24 significant bits: within tolerance
        assert_full(C, A, synth.identity(140), "f32")
    else:
        assert np.array_equal(C, A.astype(C.dtype))
    Ai = synth.small_ints(62, (150, 140))
    C = run_gemm(mmlib, Ai, synth.identity(140), _md(mmlib, mode), f64=(mode == "dgemm"))
    assert np.array_equal(C, Ai.astype(C.dtype))


@pytest.mark.parametrize("mode", MODES)
def test_diagonal(mmlib, mode):
    """The paper's diagonal special case: A.diag(d) has c_ij = a_ij d_j."""
    n = 300
    A = synth.uniform_pm1(71, (n, n))
    D = synth.diag_matrix(72, n)
    d = np.diag(D).astype(np.float64)
    C = run_gemm(mmlib, A, D, _md(mmlib, mode), f64=(mode == "dgemm"))
    exact = A.astype(np.float64) * d[None, :]
    if mode == "split":
        assert_full(C, A, D, "f32")
    elif mode == "simt":
        assert np.array_equal(C, exact.astype(np.float32))  # one rounding of an exact product
    else:
        assert np.array_equal(C, exact)


@pytest.mark.parametrize("mode", ["simt", "split"])
def test_powers_of_two_exact_reference(mmlib, mode):
    """x = +-2^k, k integer in [-20, 20]: the exact product (fixed-point
    oracle) rounded to FP32 is the reference; the paths stay within tolerance
    of it."""
    n, m, p = 96, 400, 130
    A = synth.pow2_int(81, (n, m))
    B = synth.pow2_int(82, (m, p))
    C = run_gemm(mmlib, A, B, _md(mmlib, mode))
    hi, lo = oracle.default().pow2_exact(A, B, shift=50)
    absref = np.abs(A.astype(np.float64)) @ np.abs(B.astype(np.float64))
    e = oracle.rel_errors(C, hi + lo, absref)
    assert e.max() <= oracle.tolerance(m, "f32")


@pytest.mark.parametrize("mode", ["simt", "split"])
def test_wide_exponent_rows(mmlib, mode):
    """Rows of A scaled by 2^-120 or 2^100: the per-row power-of-two scaling
    of the split path keeps the lo parts normal; both paths stay within
    tolerance."""
    n, m, p = 200, 300, 150
    e = synth.row_scale_exponents(91, n)
    A = (synth.uniform_pm1(92, (n, m)).astype(np.float64) * np.ldexp(1.0, e)[:, None]).astype(np.float32)
    B = synth.uniform_pm1(93, (m, p))
    C = run_gemm(mmlib, A, B, _md(mmlib, mode))
    assert_full(C, A, B, "f32")


def test_wide_exponent_columns_split(mmlib):
    """Columns of B scaled by 2^-120 or 2^100 (A in range): the split path
    re-packs B with its column scales and applies them in the epilogue."""
    n, m, p = 150, 2500, 190
    e = synth.row_scale_exponents(95, p)
    A = synth.uniform_pm1(96, (n, m))
    B = (synth.uniform_pm1(97, (m, p)).astype(np.float64) * np.ldexp(1.0, e)[None, :]).astype(np.float32)
    C = run_gemm(mmlib, A, B, mmlib.MM_MODE_SPLIT_BF16X3)
    assert_full(C, A, B, "f32")


def test_grouped_mixed_scaling(mmlib):
    """A grouped call where one problem needs row scales, one column scales and
    the others none: each result equals its single call and the oracle."""
    probs, host = [], []
    for g in range(6):
        n, m, p = 70 + 13 * g, 300 + 500 * g, 90 + 7 * g
        A = synth.uniform_pm1(1600 + g, (n, m))
        B = synth.uniform_pm1(1610 + g, (m, p))
        if g == 1:
            A = (A.astype(np.float64) * np.ldexp(1.0, synth.row_scale_exponents(1620, n))[:, None]).astype(np.float32)
        if g == 4:
            B = (B.astype(np.float64) * np.ldexp(1.0, synth.row_scale_exponents(1621, p))[None, :]).astype(np.float32)
        probs.append((n, m, p, dev(A), dev(B), torch.full((n, p), float("nan"), device="cuda")))
        host.append((A, B))
    assert mmlib.mm_gemm_grouped(probs, mmlib.MM_F32, mmlib.MM_MODE_SPLIT_BF16X3) == 0
    for (n, m, p, dA, dB, C), (A, B) in zip(probs, host):
        assert_full(C.cpu().numpy(), A, B, "f32")
        C1 = torch.full_like(C, float("nan"))
        assert mmlib.mm_gemm_grouped([(n, m, p, dA, dB, C1)], mmlib.MM_F32,
                                     mmlib.MM_MODE_SPLIT_BF16X3) == 0
        assert torch.equal(C, C1)
        C2 = torch.full_like(C, float("nan"))
        assert mmlib.mm_gemm(n, m, p, dA, dB, C2, mmlib.MM_F32, mmlib.MM_MODE_SPLIT_BF16X3) == 0
        assert_full(C2.cpu().numpy(), A, B, "f32")


@pytest.mark.parametrize("mode", MODES)
def test_empty_and_zero_inner(mmlib, mode):
    f64 = mode == "dgemm"
    dt = mmlib.MM_F64 if f64 else mmlib.MM_F32
    tdt = torch.float64 if f64 else torch.float32
    # m = 0: the empty sum, C = 0
    C = torch.full((5, 7), 3.0, dtype=tdt, device="cuda")
    A = torch.zeros((5, 0), dtype=tdt, device="cuda")
    B = torch.zeros((0, 7), dtype=tdt, device="cuda")
    assert mmlib.mm_gemm(5, 0, 7, A, B, C, dt, _md(mmlib, mode)) == 0
    assert torch.all(C == 0)
    # n = 0 / p = 0: nothing to do, nothing touched
    assert mmlib.mm_gemm(0, 4, 7, None, None, None, dt, _md(mmlib, mode)) == 0
    assert mmlib.mm_gemm(3, 4, 0, None, None, None, dt, _md(mmlib, mode)) == 0


@pytest.mark.parametrize("mode", MODES)
def test_transpose_identity(mmlib, mode):
    """(AB)^T = B^T A^T: the SIMT and FP64 kernels add the same products in the
    same order for both, so they agree bit for bit; the split path within
    tolerance."""
    n, m, p = 150, 333, 97
    A = synth.uniform_pm1(101, (n, m))
    B = synth.uniform_pm1(102, (m, p))
    f64 = mode == "dgemm"
    C = run_gemm(mmlib, A, B, _md(mmlib, mode), f64=f64)
    Ct = run_gemm(mmlib, B.T.copy(), A.T.copy(), _md(mmlib, mode), f64=f64)
    if mode == "split":
        assert_full(Ct.T.copy(), A, B, "f32")
    else:
        assert np.array_equal(C.T, Ct)


def test_nonfinite_propagates_simt(mmlib):
    A = synth.uniform_pm1(111, (40, 50))
    B = synth.uniform_pm1(112, (50, 60))
    A[3, 7] = np.inf
    C = run_gemm(mmlib, A, B, mmlib.MM_MODE_SIMT)
    assert not np.isfinite(C[3]).any()
    mask = np.ones(40, bool)
    mask[3] = False
    assert np.isfinite(C[mask]).all()


def test_nonfinite_split_row_becomes_nonfinite(mmlib):
    """Split path: a non-finite entry makes its row of C non-finite (NaN/inf),
    other rows stay finite and within tolerance."""
    A = synth.uniform_pm1(121, (40, 50))
    B = synth.uniform_pm1(122, (50, 60))
    A[3, 7] = np.nan
    C = run_gemm(mmlib, A, B, mmlib.MM_MODE_SPLIT_BF16X3)
    assert not np.isfinite(C[3]).any()
    mask = np.ones(40, bool)
    mask[3] = False
    assert np.isfinite(C[mask]).all()
    assert_full(C[mask], A[mask], B, "f32")
