"""Every GPU path on the stored expected values of tests/golden/, through the
C ABI: the hand-worked products (small integers: every path must give them
bit for bit, FP8 included, since the entries survive the power-of-two scaling
into e4m3 exactly) and the oracle-written seeded products (within the
elementwise tolerance; the integer case bit for bit)."""
import numpy as np
import pytest

import golden
import oracle
from gpu_util import run_gemm

pytestmark = pytest.mark.gpu

MODES = ["simt", "split", "dgemm", "fp8"]


def _md(mm, mode):
    return {"simt": mm.MM_MODE_SIMT, "split": mm.MM_MODE_SPLIT_BF16X3,
            "dgemm": mm.MM_MODE_DGEMM, "fp8": mm.MM_MODE_FP8}[mode]


@pytest.mark.parametrize("mode", MODES)
def test_hand_worked(mmlib, mode):
    for c in golden.hand_worked():
        C = run_gemm(mmlib, c["A"], c["B"], _md(mmlib, mode), f64=(mode == "dgemm"))
        assert np.array_equal(C.astype(np.float64), c["C"]), (c["name"], C)


@pytest.mark.parametrize("mode", ["simt", "split", "dgemm"])
def test_oracle_seeded(mmlib, mode):
    for c in golden.oracle_seeded():
        C = run_gemm(mmlib, c["A"], c["B"], _md(mmlib, mode), f64=(mode == "dgemm"))
        if c["name"].startswith("small_ints"):
            assert np.array_equal(C.astype(np.float64), c["C"]), c["name"]
            continue
        e = oracle.rel_errors(C.astype(np.float64), c["C"], c["ABS"])
        tol = oracle.tolerance(c["m"], "f64" if mode == "dgemm" else "f32")
        assert e.max() <= tol, (c["name"], float(e.max()), tol)
