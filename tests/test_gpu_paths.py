"""Parity of every GEMM path with the CPU oracle, element by element, at
sizes that span several tiles and ragged tails (full FP64 oracle)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import assert_full, dev, run_gemm

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 1), (1, 700, 1), (5, 1, 9), (3, 4, 5), (129, 65, 257), (300, 200, 520),
          (256, 256, 256), (1000, 37, 33), (7, 513, 1030), (257, 1024, 129), (130, 96, 70)]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("mode", ["simt", "split", "dgemm"])
def test_uniform_matches_oracle(mmlib, shape, mode):
    n, m, p = shape
    A = synth.uniform_pm1(11, (n, m))
    B = synth.uniform_pm1(12, (m, p))
    md = {"simt": mmlib.MM_MODE_SIMT, "split": mmlib.MM_MODE_SPLIT_BF16X3,
          "dgemm": mmlib.MM_MODE_DGEMM}[mode]
    C = run_gemm(mmlib, A, B, md, f64=(mode == "dgemm"))
    assert_full(C, A, B, "f64" if mode == "dgemm" else "f32")


@pytest.mark.parametrize("p", [140, 50])
@pytest.mark.parametrize("m", [1, 2, 15, 64, 2200, 2300, 3000])
def test_split_across_the_part_threshold(mmlib, m, p):
    """The split path uses three bf16 parts below m ~ 2240 and two above; both
    sides of the switch meet the tolerance, including a single-term dot
    product per entry (B with one non-zero per column).  p = 50 takes the
    64-wide N tile (a 64-row remainder in the B loads of the three-part
    split)."""
    n = 96
    A = synth.uniform_pm1(900 + m, (n, m))
    B = synth.uniform_pm1(901 + m, (m, p))
    C = run_gemm(mmlib, A, B, mmlib.MM_MODE_SPLIT_BF16X3)
    assert_full(C, A, B, "f32")
    Bs = np.zeros((m, p), np.float32)
    Bs[np.arange(p) % m, np.arange(p)] = synth.uniform_pm1(902 + m, p)
    C = run_gemm(mmlib, A, Bs, mmlib.MM_MODE_SPLIT_BF16X3)
    assert_full(C, A, Bs, "f32")


def test_config1_full_check(mmlib):
    """n = m = p = 256, entries uniform[-1,1) from seed 0 (A) / 1 (B): every
    entry of the plain SIMT kernel against the FP64 oracle."""
    A = synth.uniform_pm1(0, (256, 256))
    B = synth.uniform_pm1(1, (256, 256))
    for md in (mmlib.MM_MODE_SIMT, mmlib.MM_MODE_SPLIT_BF16X3):
        C = run_gemm(mmlib, A, B, md)
        assert_full(C, A, B, "f32")


@pytest.mark.parametrize("mode", ["simt", "split"])
def test_auto_mode(mmlib, mode):
    A = synth.uniform_pm1(21, (70, 80))
    B = synth.uniform_pm1(22, (80, 90))
    C = run_gemm(mmlib, A, B, mmlib.MM_MODE_AUTO)
    assert_full(C, A, B, "f32")
    C64 = run_gemm(mmlib, A, B, mmlib.MM_MODE_AUTO, f64=True)
    assert_full(C64, A, B, "f64")


@pytest.mark.parametrize("mode", ["simt", "split"])
def test_unaligned_operands(mmlib, mode):
    """Operands that start one element past a 16-byte boundary take the
    scalar-load variants of the same kernels."""
    md = mmlib.MM_MODE_SIMT if mode == "simt" else mmlib.MM_MODE_SPLIT_BF16X3
    n, m, p = 67, 131, 45
    A = synth.uniform_pm1(31, (n, m))
    B = synth.uniform_pm1(32, (m, p))
    bufA = torch.zeros(n * m + 1, device="cuda")
    bufB = torch.zeros(m * p + 1, device="cuda")
    bufC = torch.full((n * p + 1,), float("nan"), device="cuda")
    bufA[1:] = dev(A).reshape(-1)
    bufB[1:] = dev(B).reshape(-1)
    st = mmlib.mm_gemm(n, m, p, bufA[1:], bufB[1:], bufC[1:], mmlib.MM_F32, md)
    assert st == 0
    C = bufC[1:].reshape(n, p).cpu().numpy()
    assert_full(C, A, B, "f32")
    assert torch.isnan(bufC[0])  # nothing written before C


def test_output_untouched_outside(mmlib):
    """C is written exactly on its n x p entries: guard words around it stay."""
    n, m, p = 133, 70, 261
    A = synth.uniform_pm1(41, (n, m))
    B = synth.uniform_pm1(42, (m, p))
    for md in (mmlib.MM_MODE_SIMT, mmlib.MM_MODE_SPLIT_BF16X3):
        buf = torch.full((n * p + 64,), 7.0, device="cuda")
        st = mmlib.mm_gemm(n, m, p, dev(A), dev(B), buf[32:32 + n * p], mmlib.MM_F32, md)
        assert st == 0
        assert torch.all(buf[:32] == 7.0) and torch.all(buf[32 + n * p:] == 7.0)
        assert_full(buf[32:32 + n * p].reshape(n, p).cpu().numpy(), A, B, "f32")
