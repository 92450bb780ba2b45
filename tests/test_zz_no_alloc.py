"""The allocation-free split entry point, mm_gemm_split_static, against the
split path of mm_gemm.

Callers that cannot allocate device memory - a plug-in whose host framework
owns and accounts for all device memory, a latency-critical path that cannot
afford cudaMalloc's implicit synchronisation, a process with a fixed memory
budget - use mm_gemm_split_static: it keeps its scratch in a fixed device
array instead of allocating it.  This file is collected last so that a run
stopping at the first failure has run every other test first; it passes
alone in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import dev

pytestmark = pytest.mark.gpu


def _static_entry(mm):
    """The C entry point itself, called through ctypes."""
    fn = mm.lib().mm_gemm_split_static
    fn.argtypes = [ctypes.c_int64] * 3 + [ctypes.c_void_p] * 4
    fn.restype = ctypes.c_int
    return fn


def test_static_entry_matches_mm_gemm_twice(mmlib):
    mm = mmlib
    fn = _static_entry(mm)
    # two calls in a row: a larger product, then a smaller one that must not
    # see the first call's leftovers in the shared array
    for seed, (n, m, p) in ((1, (700, 2400, 520)), (2, (130, 300, 257))):
        A = synth.uniform_pm1(9100 + seed, (n, m))
        B = synth.uniform_pm1(9200 + seed, (m, p))
        dA, dB = dev(A), dev(B)
        C_static = torch.full((n, p), float("nan"), device="cuda")
        C_ref = torch.full((n, p), float("nan"), device="cuda")
        s = torch.cuda.current_stream()
        st = fn(n, m, p, dA.data_ptr(), dB.data_ptr(), C_static.data_ptr(), s.cuda_stream)
        assert st == mm.MM_OK, mm.mm_strerror(st)
        assert mm.mm_gemm(n, m, p, dA, dB, C_ref, mm.MM_F32, mm.MM_MODE_SPLIT_BF16X3) == 0
        cs = C_static.cpu().numpy()
        cr = C_ref.cpu().numpy()
        # against the existing entry point, in the tests' own error metric
        absref = np.abs(A.astype(np.float64)) @ np.abs(B.astype(np.float64))
        e = oracle.rel_errors(cs, cr, absref)
        assert e.max() <= oracle.tolerance(m, "f32")
        # and against the oracle
        ref, absref = oracle.default().gemm(A, B, with_abs=True)
        assert oracle.rel_errors(cs, ref, absref).max() <= oracle.tolerance(m, "f32")


def test_static_entry_rejects_oversize(mmlib):
    mm = mmlib
    fn = _static_entry(mm)
    n = 4096  # packed operands of 4096^3 exceed the fixed array
    x = torch.zeros(16, device="cuda")
    st = fn(n, n, n, x.data_ptr(), x.data_ptr(), x.data_ptr(), None)
    assert st == mm.MM_ESCRATCH
