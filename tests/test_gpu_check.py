"""The GPU FP64 check (Freivalds + sampled entries) against the oracle's own
evaluation of the same quantities."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import dev

pytestmark = pytest.mark.gpu


def _oracle_check(A, B, C, x, I, J):
    orc = oracle.default()
    y, _ = orc.gemv(C.astype(np.float64), x)
    z, za = orc.freivalds_rhs(A, B, x)
    fr = oracle.rel_errors(y, z, za).max()
    hi, lo, ab = orc.entries(A, B, I, J, "dot2")
    sm = oracle.rel_errors(C[I, J].astype(np.float64), hi + lo, ab).max()
    return fr, sm


@pytest.mark.parametrize("f64", [False, True])
def test_check_matches_oracle(mmlib, f64):
    n, m, p = 300, 257, 190
    A = synth.uniform_pm1(601, (n, m))
    B = synth.uniform_pm1(602, (m, p))
    tdt = torch.float64 if f64 else torch.float32
    # a computed product with a known perturbation in one entry
    C = (A.astype(np.float64) @ B.astype(np.float64))
    C[17, 33] += 10.0
    C = C.astype(np.float64 if f64 else np.float32)
    x = synth.freivalds_vector(603, p)
    I, J = synth.sample_indices(604, n, p, 512)
    I[0], J[0] = 17, 33
    st, fr, sm = mmlib.mm_check(n, m, p, dev(A, tdt), dev(B, tdt), dev(C), 
                                mmlib.MM_F64 if f64 else mmlib.MM_F32,
                                dev(x), dev(I), dev(J))
    assert st == 0
    ofr, osm = _oracle_check(A, B, C, x, I, J)
    assert np.isclose(fr, ofr, rtol=1e-6, atol=1e-13)
    assert np.isclose(sm, osm, rtol=1e-6, atol=1e-13)
    assert fr > 1e-5 and sm > 1e-5  # the planted error is seen by both tests


def test_check_clean_product_is_small(mmlib):
    n, m, p = 200, 300, 100
    A = synth.uniform_pm1(611, (n, m))
    B = synth.uniform_pm1(612, (m, p))
    C = torch.zeros((n, p), device="cuda")
    dA, dB = dev(A), dev(B)
    assert mmlib.mm_gemm(n, m, p, dA, dB, C, mmlib.MM_F32, mmlib.MM_MODE_SPLIT_BF16X3) == 0
    x = synth.freivalds_vector(613, p)
    I, J = synth.sample_indices(614, n, p, 256)
    st, fr, sm = mmlib.mm_check(n, m, p, dA, dB, C, mmlib.MM_F32, dev(x), dev(I), dev(J))
    assert st == 0
    tol = oracle.tolerance(m, "f32")
    assert fr <= 4 * tol and sm <= tol
    ofr, osm = _oracle_check(A, B, C.cpu().numpy(), x, I, J)
    assert np.isclose(fr, ofr, rtol=1e-6, atol=1e-13)
    assert np.isclose(sm, osm, rtol=1e-6, atol=1e-13)
