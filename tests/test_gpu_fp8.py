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
