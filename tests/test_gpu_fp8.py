"""FP8 (e4m3) path: exact on small integers (they survive the power-of-two
scaling and e4m3 rounding unchanged), and on random data its error against
the oracle is measured and reported (no tolerance is stated for it)."""
import json
import os

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import dev, run_gemm

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", [(64, 64, 64), (300, 517, 260), (129, 1000, 70)])
def test_fp8_small_integers_exact(mmlib, shape):
    """Integers in [-8, 8]: scaled by 2^4 they are multiples of 16 up to 128,
    which e4m3 holds exactly; products and FP32 sums of such integers are
    exact, so the FP8 path must give the exact integer product."""
    n, m, p = shape
    A = synth.small_ints(801, (n, m))
    B = synth.small_ints(802, (m, p))
    C = run_gemm(mmlib, A, B, mmlib.MM_MODE_FP8)
    exact = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
    assert np.array_equal(C.astype(np.float64), exact)


def test_fp8_error_reported(mmlib):
    """Uniform[-1,1) inputs: the error is that of 4-significant-bit operands
    (about 2^-5 per entry before averaging); it is recorded, and must at least
    be far below the size of the result (a sanity bound, not a tolerance)."""
    rows = []
    for n in (256, 1024):
        A = synth.uniform_pm1(811, (n, n))
        B = synth.uniform_pm1(812, (n, n))
        C = run_gemm(mmlib, A, B, mmlib.MM_MODE_FP8)
        ref, absref = oracle.default().gemm(A, B, with_abs=True)
        e = oracle.rel_errors(C, ref, absref)
        nw = oracle.normwise_error(C, ref)
        rows.append({"n": n, "e_max": float(e.max()), "e_mean": float(e.mean()),
                     "normwise": nw})
        assert e.max() < 0.05 and nw < 0.05
    out = os.environ.get("MM_REPORT_DIR")
    if out:
        with open(os.path.join(out, "fp8_error.json"), "w") as f:
            json.dump(rows, f)


def test_fp8_grouped(mmlib):
    probs = []
    for g, (n, m, p) in enumerate([(64, 300, 96), (200, 128, 33), (7, 1000, 500)]):
        A = synth.small_ints(820 + 2 * g, (n, m))
        B = synth.small_ints(821 + 2 * g, (m, p))
        probs.append((n, m, p, dev(A), dev(B), torch.zeros((n, p), device="cuda"), A, B))
    st = mmlib.mm_gemm_grouped([q[:6] for q in probs], mmlib.MM_F32, mmlib.MM_MODE_FP8)
    assert st == 0
    for (n, m, p, _, _, C, A, B) in probs:
        exact = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float32)
        assert np.array_equal(C.cpu().numpy(), exact)


def test_fp8_block_scales_keep_small_blocks(mmlib):
    """Scales per 128-value K block: a row whose first block holds values near
    2^30 and whose other blocks hold values near 1 keeps the small blocks'
    significance (one scale per row would push them below the e4m3 range and
    lose them).  Here the small blocks carry most of |A||B| for the columns of
    B that are zero on the first block, so one scale per row would give an
    error near 1 there; per block it is that of 4-bit operands."""
    n, m, p = 130, 640, 70
    A = synth.uniform_pm1(831, (n, m)).astype(np.float64)
    A[:, :128] *= 2.0 ** 30
    B = synth.uniform_pm1(832, (m, p)).astype(np.float64)
    B[:128, : p // 2] = 0.0  # half of the columns never meet the large block
    A = A.astype(np.float32)
    B = B.astype(np.float32)
    C = run_gemm(mmlib, A, B, mmlib.MM_MODE_FP8)
    ref, absref = oracle.default().gemm(A, B, with_abs=True)
    e = oracle.rel_errors(C, ref, absref)
    assert np.isfinite(C).all()
    assert e.max() < 0.05, e.max()
    assert e[:, : p // 2].max() < 0.05


@pytest.mark.parametrize("shape", [(1, 1, 1), (5, 129, 3), (257, 300, 130), (128, 128, 128)])
def test_fp8_ragged_shapes(mmlib, shape):
    """Edges of the 128 x 128 tiles and of the 128-value K blocks (zero
    padding), against the oracle within the e4m3 sanity bound."""
    n, m, p = shape
    A = synth.uniform_pm1(841, (n, m))
    B = synth.uniform_pm1(842, (m, p))
    C = run_gemm(mmlib, A, B, mmlib.MM_MODE_FP8)
    ref, absref = oracle.default().gemm(A, B, with_abs=True)
    assert oracle.rel_errors(C, ref, absref).max() < 0.05


def test_fp8_grouped_equals_single(mmlib):
    """A grouped call runs the same kernels with the same per-block scales:
    each product's bits equal its single call."""
    probs, host = [], []
    for g, (n, m, p) in enumerate([(100, 300, 96), (260, 1000, 140), (7, 129, 500)]):
        A = synth.uniform_pm1(850 + 2 * g, (n, m))
        B = synth.uniform_pm1(851 + 2 * g, (m, p))
        probs.append((n, m, p, dev(A), dev(B), torch.full((n, p), float("nan"), device="cuda")))
        host.append((A, B))
    assert mmlib.mm_gemm_grouped(probs, mmlib.MM_F32, mmlib.MM_MODE_FP8) == 0
    for (n, m, p, dA, dB, C), (A, B) in zip(probs, host):
        C1 = torch.full_like(C, float("nan"))
        assert mmlib.mm_gemm(n, m, p, dA, dB, C1, mmlib.MM_F32, mmlib.MM_MODE_FP8) == 0
        assert torch.equal(C, C1), (n, m, p)


def test_fp8_uniform_and_blockwise_tiles_in_one_product(mmlib):
    """Tiles whose rows and columns keep one exponent along K accumulate all K
    blocks in tensor memory and are unscaled once; the others unscale each K
    block.  One product with both kinds (row tile 0 of A has one K block
    scaled by 2^12, so its tiles take the blockwise form): every tile within
    the e4m3 sanity bound of the oracle, and the blockwise tiles' rows equal
    to a product of those rows alone (the same decision per tile)."""
    n, m, p = 256, 512, 256
    A = synth.uniform_pm1(861, (n, m)).astype(np.float64)
    A[:128, 128:256] *= 2.0 ** 12
    A = A.astype(np.float32)
    B = synth.uniform_pm1(862, (m, p))
    C = run_gemm(mmlib, A, B, mmlib.MM_MODE_FP8)
    ref, absref = oracle.default().gemm(A, B, with_abs=True)
    e = oracle.rel_errors(C, ref, absref)
    assert e[:128].max() < 0.05 and e[128:].max() < 0.05, (e[:128].max(), e[128:].max())
    C0 = run_gemm(mmlib, np.ascontiguousarray(A[:128]), B, mmlib.MM_MODE_FP8)
    assert np.array_equal(C0, C[:128])
    C1 = run_gemm(mmlib, np.ascontiguousarray(A[128:]), B, mmlib.MM_MODE_FP8)
    assert np.array_equal(C1, C[128:])
