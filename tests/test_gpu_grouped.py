"""Grouped GEMM: uneven independent products in one launch per path, each
result against the oracle."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import dev

pytestmark = pytest.mark.gpu


def _problems(count, seed, lo=32, hi=1024, step=32, f64=False):
    dims = synth.grouped_dims(seed, count, lo, hi, step)
    tdt = torch.float64 if f64 else torch.float32
    probs, host = [], []
    for g, (n, m, p) in enumerate(dims):
        A = synth.uniform_pm1(1000 + 2 * g, (n, m))
        B = synth.uniform_pm1(1001 + 2 * g, (m, p))
        C = torch.full((n, p), float("nan"), dtype=tdt, device="cuda")
        probs.append((int(n), int(m), int(p), dev(A, tdt), dev(B, tdt), C))
        host.append((A, B))
    return probs, host


@pytest.mark.parametrize("mode", ["split", "simt", "dgemm"])
def test_grouped_uneven(mmlib, mode):
    f64 = mode == "dgemm"
    md = {"split": mmlib.MM_MODE_SPLIT_BF16X3, "simt": mmlib.MM_MODE_SIMT,
          "dgemm": mmlib.MM_MODE_DGEMM}[mode]
    probs, host = _problems(24, 7, lo=1, hi=700, step=1, f64=f64)
    st = mmlib.mm_gemm_grouped(probs, mmlib.MM_F64 if f64 else mmlib.MM_F32, md)
    assert st == 0, mmlib.mm_strerror(st)
    orc = oracle.default()
    for (n, m, p, _, _, C), (A, B) in zip(probs, host):
        ref, absref = orc.gemm(A, B, with_abs=True)
        e = oracle.rel_errors(C.cpu().numpy(), ref, absref).max()
        assert e <= oracle.tolerance(m, "f64" if f64 else "f32"), (n, m, p, e)


def test_grouped_matches_single(mmlib):
    """Each grouped result equals the same product run alone as a grouped call
    of one (same tiles, same tail split), and mm_gemm's result (the fused
    split-K kernel for products with few tiles) within the tolerance."""
    probs, host = _problems(12, 9)
    assert mmlib.mm_gemm_grouped(probs, mmlib.MM_F32, mmlib.MM_MODE_SPLIT_BF16X3) == 0
    for (n, m, p, A, B, C), (Ah, Bh) in zip(probs, host):
        C1 = torch.full_like(C, float("nan"))
        assert mmlib.mm_gemm_grouped([(n, m, p, A, B, C1)], mmlib.MM_F32,
                                     mmlib.MM_MODE_SPLIT_BF16X3) == 0
        bn_g = mmlib.mm_tune_query(n, m, p)[1]
        assert torch.equal(C, C1), (n, m, p, bn_g)
        C2 = torch.full_like(C, float("nan"))
        assert mmlib.mm_gemm(n, m, p, A, B, C2, mmlib.MM_F32, mmlib.MM_MODE_SPLIT_BF16X3) == 0
        absref = np.abs(Ah.astype(np.float64)) @ np.abs(Bh.astype(np.float64))
        e = oracle.rel_errors(C2.cpu().numpy(), C1.cpu().numpy(), absref).max()
        assert e <= oracle.tolerance(m, "f32"), (n, m, p, e)


def test_grouped_config4_full(mmlib):
    """The config-4 workload as the bench runs it: 4096 instances, n, m, p
    uniform over {32, 64, ..., 1024} (seed 4), seeded uniform[-1,1) operands,
    one grouped call.  Every instance passes the library's FP64 GPU check
    (one Freivalds vector and 64 sampled entries against 1e-6 sqrt(m)), and 64
    instances (every 64th) are compared with the CPU oracle in full."""
    dims = synth.grouped_dims(4, 4096)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(4)
    probs = []
    for (n, m, p) in dims:
        n, m, p = int(n), int(m), int(p)
        A = torch.rand((n, m), device="cuda", generator=gen) * 2 - 1
        B = torch.rand((m, p), device="cuda", generator=gen) * 2 - 1
        probs.append((n, m, p, A, B, torch.full((n, p), float("nan"), device="cuda")))
    assert mmlib.mm_gemm_grouped(probs, mmlib.MM_F32, mmlib.MM_MODE_SPLIT_BF16X3) == 0
    chk = torch.Generator(device="cuda")
    worst = 0.0
    for g, (n, m, p, A, B, C) in enumerate(probs):
        chk.manual_seed(100 + g)
        x = torch.rand(p, device="cuda", dtype=torch.float64, generator=chk) * 2 - 1
        I = torch.randint(0, n, (64,), device="cuda", generator=chk)
        J = torch.randint(0, p, (64,), device="cuda", generator=chk)
        st, fr, sm = mmlib.mm_check(n, m, p, A, B, C, mmlib.MM_F32, x, I, J)
        assert st == mmlib.MM_OK
        e = max(fr, sm) / oracle.tolerance(m, "f32")
        assert e <= 1.0, (g, n, m, p, fr, sm)
        worst = max(worst, e)
    orc = oracle.default()
    for g in range(0, 4096, 64):
        n, m, p, A, B, C = probs[g]
        ref, absref = orc.gemm(A.cpu().numpy(), B.cpu().numpy(), with_abs=True)
        e = oracle.rel_errors(C.cpu().numpy(), ref, absref).max()
        assert e <= oracle.tolerance(m, "f32"), (g, n, m, p, e)


def test_grouped_config4_sample(mmlib):
    """Config-4 shape mix (n, m, p uniform over {32, 64, ..., 1024}): 256 of
    the instances (synth operands) in one launch, every 8th compared with the
    oracle in full."""
    probs, host = _problems(256, 4)
    assert mmlib.mm_gemm_grouped(probs, mmlib.MM_F32, mmlib.MM_MODE_SPLIT_BF16X3) == 0
    orc = oracle.default()
    for g in range(0, 256, 8):
        n, m, p, _, _, C = probs[g]
        A, B = host[g]
        ref, absref = orc.gemm(A, B, with_abs=True)
        e = oracle.rel_errors(C.cpu().numpy(), ref, absref).max()
        assert e <= oracle.tolerance(m, "f32"), (g, n, m, p, e)


def test_grouped_with_empty_members(mmlib):
    A = torch.ones((3, 0), device="cuda")
    B = torch.ones((0, 4), device="cuda")
    C = torch.full((3, 4), 5.0, device="cuda")
    A2 = dev(synth.uniform_pm1(1, (40, 50)))
    B2 = dev(synth.uniform_pm1(2, (50, 30)))
    C2 = torch.zeros((40, 30), device="cuda")
    probs = [(3, 0, 4, A, B, C), (0, 5, 5, None, None, None), (40, 50, 30, A2, B2, C2)]
    assert mmlib.mm_gemm_grouped(probs, mmlib.MM_F32, mmlib.MM_MODE_SPLIT_BF16X3) == 0
    assert torch.all(C == 0)
    a2 = synth.uniform_pm1(1, (40, 50))
    b2 = synth.uniform_pm1(2, (50, 30))
    ref, absref = oracle.default().gemm(a2, b2, with_abs=True)
    assert oracle.rel_errors(C2.cpu().numpy(), ref, absref).max() <= oracle.tolerance(50, "f32")
