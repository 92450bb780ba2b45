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
from gpu_util import dev, fused_slices

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


def test_static_entry_rescaled_rows_then_uniform(mmlib):
    """Rows of A at 2^-120 and 2^100 make the verify pass flag A and the fix
    pass re-pack it with its scales; the next call, on plain uniform data,
    must start from cleared flags in the shared array."""
    mm = mmlib
    fn = _static_entry(mm)
    s = torch.cuda.current_stream()
    n, m, p = 300, 700, 260
    A = synth.uniform_pm1(9301, (n, m))
    A = (A.astype(np.float64) * np.ldexp(1.0, synth.row_scale_exponents(9302, n))[:, None]
         ).astype(np.float32)
    B = synth.uniform_pm1(9303, (m, p))
    A2 = synth.uniform_pm1(9304, (n, m))
    orc = oracle.default()
    for a in (A, A2):
        dA, dB = dev(a), dev(B)
        C = torch.full((n, p), float("nan"), device="cuda")
        st = fn(n, m, p, dA.data_ptr(), dB.data_ptr(), C.data_ptr(), s.cuda_stream)
        assert st == mm.MM_OK, mm.mm_strerror(st)
        ref, absref = orc.gemm(a, B, with_abs=True)
        e = oracle.rel_errors(C.cpu().numpy(), ref, absref)
        assert e.max() <= oracle.tolerance(m, "f32"), e.max()


def test_static_entry_bitwise_where_no_tail_split(mmlib):
    """Where mm_gemm neither splits its last wave along K nor runs the product
    on the fused split-K kernel, both entry points run the same kernels with
    the same tiles, so the bits agree."""
    mm = mmlib
    fn = _static_entry(mm)
    s = torch.cuda.current_stream()
    checked = 0
    for seed, (n, m, p) in enumerate(((2432, 512, 2048), (2560, 2300, 1024), (1000, 1500, 900))):
        st, tiles, split_from, split_s = mm.mm_tune_query_tail(n, m, p)
        assert st == mm.MM_OK
        if split_s > 1 or fused_slices(mm, n, m, p) > 0:
            continue
        A = synth.uniform_pm1(9400 + seed, (n, m))
        B = synth.uniform_pm1(9500 + seed, (m, p))
        dA, dB = dev(A), dev(B)
        C1 = torch.full((n, p), float("nan"), device="cuda")
        C2 = torch.full((n, p), float("nan"), device="cuda")
        st = fn(n, m, p, dA.data_ptr(), dB.data_ptr(), C1.data_ptr(), s.cuda_stream)
        assert st == mm.MM_OK, mm.mm_strerror(st)
        assert mm.mm_gemm(n, m, p, dA, dB, C2, mm.MM_F32, mm.MM_MODE_SPLIT_BF16X3) == 0
        assert torch.equal(C1.view(torch.int32), C2.view(torch.int32)), (n, m, p)
        checked += 1
    assert checked >= 1


def test_static_entry_rejects_oversize(mmlib):
    mm = mmlib
    fn = _static_entry(mm)
    n = 4096  # packed operands of 4096^3 exceed the fixed array
    x = torch.zeros(16, device="cuda")
    st = fn(n, n, n, x.data_ptr(), x.data_ptr(), x.data_ptr(), None)
    assert st == mm.MM_ESCRATCH
