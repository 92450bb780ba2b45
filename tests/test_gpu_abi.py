"""Boundary behaviour through the C ABI: status codes, host operands,
asynchronous calls, tracing, tuner table round trip."""
import os

import numpy as np
import pytest
import torch

import oracle
from gpu_util import fused_slices
import synth
from gpu_util import assert_full, dev

pytestmark = pytest.mark.gpu


def test_status_codes(mmlib):
    mm = mmlib
    x = torch.zeros(16, device="cuda")
    assert mm.mm_init(device=0) == mm.MM_EBUSY
    assert mm.mm_gemm(-1, 2, 2, x, x, x, mm.MM_F32, mm.MM_MODE_SIMT) == mm.MM_EINVAL
    assert mm.mm_gemm(2, 2, 2, None, x, x, mm.MM_F32, mm.MM_MODE_SIMT) == mm.MM_EINVAL
    assert mm.mm_gemm(2, 2, 2, x, x, None, mm.MM_F32, mm.MM_MODE_SIMT) == mm.MM_EINVAL
    assert mm.mm_gemm(2, 2, 2, x, x, x, mm.MM_F64, mm.MM_MODE_SIMT) == mm.MM_EUNSUPPORTED
    assert mm.mm_gemm(2, 2, 2, x, x, x, mm.MM_F64, mm.MM_MODE_SPLIT_BF16X3) == mm.MM_EUNSUPPORTED
    assert mm.mm_gemm(2, 2, 2, x, x, x, mm.MM_F32, mm.MM_MODE_DGEMM) == mm.MM_EUNSUPPORTED
    assert mm.mm_gemm(2, 2, 2, x, x, x, 7, mm.MM_MODE_SIMT) == mm.MM_EINVAL
    assert mm.mm_gemm(2, 2, 2, x, x, x, mm.MM_F32, 9) == mm.MM_EINVAL
    # async entry points take device memory only
    h = np.zeros(16, np.float32)
    assert mm.mm_gemm_async(2, 2, 2, h, x, x, mm.MM_F32, mm.MM_MODE_SIMT) == mm.MM_EINVAL
    st, rid = mm.mm_poll(123456789)[0], None
    assert st in (mm.MM_ENOTFOUND,)


def test_shutdown_is_idempotent_and_reinit(mmlib):
    mm = mmlib
    assert mm.mm_shutdown() == mm.MM_OK
    assert mm.mm_shutdown() == mm.MM_OK
    x = torch.zeros(4, device="cuda")
    assert mm.mm_gemm(1, 1, 1, x, x, x, mm.MM_F32, mm.MM_MODE_SIMT) == mm.MM_ENOTINIT
    assert mm.mm_init(device=0) == mm.MM_OK


@pytest.mark.parametrize("mode", ["simt", "split", "dgemm"])
def test_host_operands(mmlib, mode):
    """mm_gemm with host (numpy) operands stages them through the library."""
    mm = mmlib
    f64 = mode == "dgemm"
    md = {"simt": mm.MM_MODE_SIMT, "split": mm.MM_MODE_SPLIT_BF16X3, "dgemm": mm.MM_MODE_DGEMM}[mode]
    n, m, p = 90, 130, 75
    A = synth.uniform_pm1(701, (n, m))
    B = synth.uniform_pm1(702, (m, p))
    dtp = np.float64 if f64 else np.float32
    Ah, Bh = A.astype(dtp), B.astype(dtp)
    Ch = np.full((n, p), np.nan, dtp)
    st = mm.mm_gemm(n, m, p, Ah, Bh, Ch, mm.MM_F64 if f64 else mm.MM_F32, md)
    assert st == 0
    assert_full(Ch, A, B, "f64" if f64 else "f32")
    # pinned host memory, mixed with a device output
    Ap = torch.from_numpy(Ah).pin_memory()
    Cd = torch.full((n, p), float("nan"), dtype=torch.float64 if f64 else torch.float32,
                    device="cuda")
    st = mm.mm_gemm(n, m, p, Ap, dev(Bh), Cd, mm.MM_F64 if f64 else mm.MM_F32, md)
    assert st == 0
    assert_full(Cd.cpu().numpy(), A, B, "f64" if f64 else "f32")


@pytest.mark.parametrize("shape", [(2304, 700, 300), (4100, 2500, 129), (4100, 2500, 2000)])
def test_host_operands_pipelined(mmlib, shape):
    """Large host-operand split products go through the slab pipeline (B
    packed once, rows of A in slabs, copies overlapping the tensor cores);
    the result is identical to the device-operand call where that call does
    not split its last wave of tiles along K (the slabs never do), else
    within the tolerance of it."""
    mm = mmlib
    n, m, p = shape
    A = synth.uniform_pm1(731, (n, m))
    B = synth.uniform_pm1(732, (m, p))
    Ap = torch.from_numpy(A).pin_memory()
    Bp = torch.from_numpy(B).pin_memory()
    Cp = torch.full((n, p), float("nan")).pin_memory()
    assert mm.mm_gemm(n, m, p, Ap, Bp, Cp, mm.MM_F32, mm.MM_MODE_SPLIT_BF16X3) == 0
    Cd = torch.full((n, p), float("nan"), device="cuda")
    assert mm.mm_gemm(n, m, p, dev(A), dev(B), Cd, mm.MM_F32, mm.MM_MODE_SPLIT_BF16X3) == 0
    st, _, _, split_s = mm.mm_tune_query_tail(n, m, p)
    assert st == 0
    if split_s == 1 and fused_slices(mm, n, m, p) == 0:
        assert torch.equal(Cp, Cd.cpu())
    else:
        absref = np.abs(A.astype(np.float64)) @ np.abs(B.astype(np.float64))
        e = oracle.rel_errors(Cp.numpy(), Cd.cpu().numpy().astype(np.float64), absref)
        assert e.max() <= oracle.tolerance(m, "f32")
    from gpu_util import sampled_check
    sampled_check(Cp.numpy(), A, B, "f32", count=1024, trials=1)


def test_async_on_torch_stream_and_trace(mmlib):
    """Queued calls on a caller stream and the launch tracer: a product with
    enough tiles for the packed path launches its four kernels per call; one
    with few tiles launches the fused split-K kernel once per call."""
    mm = mmlib
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    n, m, p = 128 * n_sm, 384, 640
    A = synth.uniform_pm1(711, (n, m))
    B = synth.uniform_pm1(712, (m, p))
    dA, dB = dev(A), dev(B)
    C = torch.full((n, p), float("nan"), device="cuda")
    s = torch.cuda.Stream()
    mm.mm_trace_reset()
    assert mm.mm_trace_enable(True) == 0
    before = mm.mm_launch_count()
    for _ in range(3):
        assert mm.mm_gemm_async(n, m, p, dA, dB, C, mm.MM_F32, mm.MM_MODE_SPLIT_BF16X3, s) == 0
    assert mm.mm_sync(s) == 0
    # unscaled pack + verify + re-pack of flagged operands + tensor core, 3 times
    assert mm.mm_launch_count() - before == 12
    st, k, ms = mm.mm_trace_read("split_tc")
    assert st == 0 and k == 3 and ms > 0
    st, k, _ = mm.mm_trace_read("split_pack")
    assert k == 3
    mm.mm_trace_reset()
    assert_full(C.cpu().numpy(), A, B, "f32")
    n2, m2, p2 = 512, 384, 640
    assert fused_slices(mm, n2, m2, p2) > 0
    C2 = torch.full((n2, p2), float("nan"), device="cuda")
    before = mm.mm_launch_count()
    for _ in range(3):
        assert mm.mm_gemm_async(n2, m2, p2, dA[:n2], dB, C2, mm.MM_F32, mm.MM_MODE_SPLIT_BF16X3,
                                s) == 0
    assert mm.mm_sync(s) == 0
    assert mm.mm_launch_count() - before == 3
    st, k, ms = mm.mm_trace_read("fused_tc")
    assert st == 0 and k == 3 and ms > 0
    mm.mm_trace_enable(False)
    mm.mm_trace_reset()
    assert_full(C2.cpu().numpy(), A[:n2], B, "f32")


def test_tune_table_roundtrip(mmlib, tmp_path):
    mm = mmlib
    assert mm.mm_tune(256, 512, 384, 2) == 0
    st, bn, bk, stages, gm = mm.mm_tune_query(256, 512, 384)
    assert st == 0 and bn in (128, 256) and bk in (32, 64)
    path = str(tmp_path / "tune.txt")
    assert mm.mm_tune_save(path) == 0
    text = open(path).read()
    # buckets are ceil(log2) of each size: 256 -> 8, 512 -> 9, 384 -> 9
    assert "%d %d %d %d" % (8, 9, 9, bn) in text
    bad = tmp_path / "bad.txt"
    bad.write_text("9 9 9 100 32 4 8 0\n")
    assert mm.mm_tune_load(str(bad)) == mm.MM_EINVAL
    assert mm.mm_tune_load(path) == 0
    # results with the tuned choice still match the oracle
    A = synth.uniform_pm1(721, (256, 512))
    B = synth.uniform_pm1(722, (512, 384))
    C = torch.zeros((256, 384), device="cuda")
    assert mm.mm_gemm(256, 512, 384, dev(A), dev(B), C, mm.MM_F32, mm.MM_MODE_SPLIT_BF16X3) == 0
    assert_full(C.cpu().numpy(), A, B, "f32")


def test_measure_fma_peak(mmlib):
    """The CUDA cores' measured FMA rates: FP32 near 128 FMAs per SM and clock
    (80 TFLOP/s at 2.07 GHz on 152 SMs), FP64 far lower on this part."""
    mm = mmlib
    st, f32 = mm.mm_measure_fma_peak(mm.MM_F32, 2048)
    assert st == mm.MM_OK and 30e12 < f32 < 120e12, f32
    st, f64 = mm.mm_measure_fma_peak(mm.MM_F64, 64)
    assert st == mm.MM_OK and 0.05e12 < f64 < f32, f64
    assert mm.mm_measure_fma_peak(mm.MM_F32, 0)[0] == mm.MM_EINVAL
