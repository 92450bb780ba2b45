"""SIMT FP32 and FP64 products with too few output tiles for the SMs (skinny
and small ones): mm_gemm cuts K into slices, computes each slice's partial
product on 64 x 64 tiles and adds the partials in a fixed order in a second
kernel.  Checked against the CPU oracle in full, exact on small integers,
deterministic, and the same bit for bit for (AB)^T and B^T A^T; the two-kernel
form is confirmed through the library's launch counter."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import assert_full, dev, run_gemm

pytestmark = pytest.mark.gpu


def _launches(mm, fn):
    fn()
    torch.cuda.synchronize()
    l0 = mm.mm_launch_count()
    fn()
    torch.cuda.synchronize()
    return mm.mm_launch_count() - l0


@pytest.mark.parametrize("shape", [(64, 16384, 64), (70, 4999, 33), (1, 3000, 1), (200, 2048, 150),
                                   (1024, 1024, 1024)])
def test_simt_splitk_against_oracle(mmlib, shape):
    """Skinny (the config-3 shape), ragged with K not a multiple of 4 (the
    unaligned loads), one entry, and a product of a few tiles; FP32 and FP64."""
    n, m, p = shape
    A = synth.uniform_pm1(5200 + n, (n, m))
    B = synth.uniform_pm1(5201 + p, (m, p))
    C = run_gemm(mmlib, A, B, mmlib.MM_MODE_SIMT)
    assert_full(C, A, B, "f32")
    A64 = synth.uniform_pm1_f64(5202 + n, (n, m))
    B64 = synth.uniform_pm1_f64(5203 + p, (m, p))
    C64 = run_gemm(mmlib, A64, B64, mmlib.MM_MODE_DGEMM, f64=True)
    assert_full(C64, A64, B64, "f64")


def test_simt_splitk_runs_two_kernels(mmlib):
    """The skinny product takes the slices and the fixed-order sum (two
    launches); a square product that fills the SMs keeps one launch."""
    mm = mmlib
    for (n, m, p), want in (((64, 16384, 64), 2), ((2048, 512, 2048), 1)):
        A = dev(synth.uniform_pm1(5300, (n, m)))
        B = dev(synth.uniform_pm1(5301, (m, p)))
        C = torch.empty((n, p), device="cuda")
        got = _launches(mm, lambda: mm.mm_gemm(n, m, p, A, B, C, mm.MM_F32, mm.MM_MODE_SIMT))
        assert got == want, ((n, m, p), got)


def test_simt_splitk_small_integers_exact(mmlib):
    """Integer entries in [-8, 8]: every partial and every sum is exact, so the
    sliced sum equals the integer product bit for bit."""
    A = synth.small_ints(5400, (65, 6000)).astype(np.float64)
    B = synth.small_ints(5401, (6000, 40)).astype(np.float64)
    exact = A.astype(np.int64) @ B.astype(np.int64)
    C = run_gemm(mmlib, A.astype(np.float32), B.astype(np.float32), mmlib.MM_MODE_SIMT)
    assert np.array_equal(C.astype(np.int64), exact)
    C64 = run_gemm(mmlib, A, B, mmlib.MM_MODE_DGEMM, f64=True)
    assert np.array_equal(C64.astype(np.int64), exact)


def test_simt_splitk_deterministic_and_transpose(mmlib):
    """The slices and their order depend on the shape only: two calls give the
    same bits, and (AB)^T = B^T A^T bit for bit (the same products, the same
    slices, the same order)."""
    n, m, p = 96, 7000, 40
    A = synth.uniform_pm1(5500, (n, m))
    B = synth.uniform_pm1(5501, (m, p))
    for md, f64 in ((mmlib.MM_MODE_SIMT, False), (mmlib.MM_MODE_DGEMM, True)):
        a, b = (A, B) if not f64 else (A.astype(np.float64), B.astype(np.float64))
        C1 = run_gemm(mmlib, a, b, md, f64=f64)
        C2 = run_gemm(mmlib, a, b, md, f64=f64)
        assert np.array_equal(C1, C2)
        Ct = run_gemm(mmlib, b.T.copy(), a.T.copy(), md, f64=f64)
        assert np.array_equal(C1.T, Ct)


def test_simt_splitk_nonfinite(mmlib):
    """An infinity in a row of A makes that row of C non-finite through the
    slices' sum, and leaves the other rows finite."""
    A = synth.uniform_pm1(5600, (40, 9000))
    B = synth.uniform_pm1(5601, (9000, 30))
    A[3, 8000] = np.inf
    C = run_gemm(mmlib, A, B, mmlib.MM_MODE_SIMT)
    assert not np.isfinite(C[3]).any()
    rest = np.delete(C, 3, axis=0)
    assert np.isfinite(rest).all()
    ref, ab = oracle.default().gemm(np.delete(A, 3, axis=0), B, with_abs=True)
    assert oracle.rel_errors(rest, ref, ab).max() <= oracle.tolerance(9000, "f32")
