"""Parity at the full workload sizes (square 1024..8192, rectangular, skinny,
diagonal, wide exponents) on 4096 sampled entries plus two Freivalds trials,
in the launch configuration the benchmark times; the square sizes up to 2048
also against the oracle's full product."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import dev, sampled_check

pytestmark = pytest.mark.gpu


def _run(mm, A, B, mode, f64=False):
    n, m = A.shape
    p = B.shape[1]
    tdt = torch.float64 if f64 else torch.float32
    dC = torch.full((n, p), float("nan"), dtype=tdt, device="cuda")
    st = mm.mm_gemm(n, m, p, dev(A, tdt), dev(B, tdt), dC, mm.MM_F64 if f64 else mm.MM_F32, mode)
    assert st == 0, mm.mm_strerror(st)
    C = dC.cpu().numpy()
    del dC
    return C


@pytest.mark.parametrize("n", [1024, 2048, 4096, 8192])
def test_square_f32_paths(mmlib, n):
    """Sampled entries and Freivalds at every size; at n <= 2048 also every
    entry against the oracle's full product."""
    A = synth.uniform_pm1(2 * n, (n, n))
    B = synth.uniform_pm1(2 * n + 1, (n, n))
    full = oracle.default().gemm(A, B, with_abs=True) if n <= 2048 else None
    for mode in (mmlib.MM_MODE_SPLIT_BF16X3, mmlib.MM_MODE_SIMT):
        C = _run(mmlib, A, B, mode)
        sampled_check(C, A, B, "f32")
        if full is not None:
            e = oracle.rel_errors(C, *full).max()
            assert e <= oracle.tolerance(n, "f32"), (mode, e)


@pytest.mark.parametrize("n", [1024, 4096, 8192])
def test_square_dgemm(mmlib, n):
    A = synth.uniform_pm1(2 * n, (n, n))
    B = synth.uniform_pm1(2 * n + 1, (n, n))
    C = _run(mmlib, A, B, mmlib.MM_MODE_DGEMM, f64=True)
    sampled_check(C, A, B, "f64")
    if n <= 2048:
        e = oracle.rel_errors(C, *oracle.default().gemm(A, B, with_abs=True)).max()
        assert e <= oracle.tolerance(n, "f64"), e


@pytest.mark.parametrize("shape", [(8192, 512, 8192), (64, 16384, 64)], ids=["rect", "skinny"])
def test_stress_shapes(mmlib, shape):
    n, m, p = shape
    A = synth.uniform_pm1(301, (n, m))
    B = synth.uniform_pm1(302, (m, p))
    for mode in (mmlib.MM_MODE_SPLIT_BF16X3, mmlib.MM_MODE_SIMT):
        C = _run(mmlib, A, B, mode)
        sampled_check(C, A, B, "f32")


def test_diagonal_4096(mmlib):
    n = 4096
    A = synth.uniform_pm1(401, (n, n))
    D = synth.diag_matrix(402, n)
    d = np.diag(D).astype(np.float64)
    exact = (A.astype(np.float64) * d[None, :])
    C = _run(mmlib, A, D, mmlib.MM_MODE_SIMT)
    assert np.array_equal(C, exact.astype(np.float32))
    C = _run(mmlib, A, D, mmlib.MM_MODE_SPLIT_BF16X3)
    sampled_check(C, A, D, "f32")


def test_pow2_real_exponents_4096(mmlib):
    """Entries s * 2^e, e uniform real in [-20, 20): 40 binades per operand."""
    n = 4096
    A = synth.pow2_real(501, (n, n))
    B = synth.pow2_real(502, (n, n))
    for mode in (mmlib.MM_MODE_SPLIT_BF16X3, mmlib.MM_MODE_SIMT):
        C = _run(mmlib, A, B, mode)
        sampled_check(C, A, B, "f32")
