"""The split ladder: MM_MODE_SPLIT_BF16X6 (three bf16 parts, six products) as
a mode of its own, against the CPU oracle at every size, and its accuracy
against the two-part SPLIT_BF16X3 on the same inputs."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_full, full_errors, run_gemm

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 1), (3, 4, 5), (129, 65, 257), (300, 2300, 200), (257, 4096, 129),
          (1000, 37, 33), (7, 513, 1030)]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_x6_matches_oracle(mmlib, shape):
    n, m, p = shape
    A = synth.uniform_pm1(61, (n, m))
    B = synth.uniform_pm1(62, (m, p))
    C = run_gemm(mmlib, A, B, mmlib.MM_MODE_SPLIT_BF16X6)
    assert_full(C, A, B, "f32")


def test_x6_more_accurate_than_x3_where_the_split_dominates(mmlib):
    """With one non-zero term per output (B holds one entry per column) the
    two-part split leaves up to 3 2^-16 of the term, the three-part split about
    2^-24.  On dense uniform data at the same m = 4096 both errors come from
    the tensor cores' FP32 accumulation of thousands of products and are of the
    same size (measured on GB300: 4.7e-7 and 6.1e-7 of |A||B|), both far within
    the tolerance."""
    n, m, p = 256, 4096, 256
    A = synth.uniform_pm1(63, (n, m))
    Bs = np.zeros((m, p), np.float32)
    Bs[(np.arange(p) * 13) % m, np.arange(p)] = synth.uniform_pm1(64, p)
    e3, _ = full_errors(run_gemm(mmlib, A, Bs, mmlib.MM_MODE_SPLIT_BF16X3), A, Bs)
    e6, _ = full_errors(run_gemm(mmlib, A, Bs, mmlib.MM_MODE_SPLIT_BF16X6), A, Bs)
    tol = oracle.tolerance(m, "f32")
    assert e3.max() <= tol and e6.max() <= tol
    assert e6.max() * 64 < e3.max(), (e6.max(), e3.max())
    B = synth.uniform_pm1(64, (m, p))
    e3, _ = full_errors(run_gemm(mmlib, A, B, mmlib.MM_MODE_SPLIT_BF16X3), A, B)
    e6, _ = full_errors(run_gemm(mmlib, A, B, mmlib.MM_MODE_SPLIT_BF16X6), A, B)
    assert e3.max() <= tol and e6.max() <= tol
    assert e6.max() <= 4 * e3.max(), (e6.max(), e3.max())


def test_x6_small_integers_exact(mmlib):
    n, m, p = 100, 3000, 90
    A = synth.small_ints(65, (n, m))
    B = synth.small_ints(66, (m, p))
    C = run_gemm(mmlib, A, B, mmlib.MM_MODE_SPLIT_BF16X6)
    exact = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float32)
    assert np.array_equal(C, exact)


def test_x6_rescaled_rows(mmlib):
    """Rows of A at 2^-120 / 2^100: the fix pass re-packs the three parts with
    their power-of-two scales."""
    n, m, p = 140, 700, 90
    A = synth.uniform_pm1(67, (n, m))
    A = (A.astype(np.float64) * np.ldexp(1.0, synth.row_scale_exponents(68, n))[:, None]
         ).astype(np.float32)
    B = synth.uniform_pm1(69, (m, p))
    C = run_gemm(mmlib, A, B, mmlib.MM_MODE_SPLIT_BF16X6)
    assert_full(C, A, B, "f32")


def test_x6_rejects_f64(mmlib):
    import torch
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    st = mmlib.mm_gemm(2, 2, 1, x, x, x, mmlib.MM_F64, mmlib.MM_MODE_SPLIT_BF16X6)
    assert st == mmlib.MM_EUNSUPPORTED
