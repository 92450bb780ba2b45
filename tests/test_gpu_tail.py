"""Tail split of the tensor-core path.

When a single product's 128 x bn tiles leave the last wave of the persistent
grid partly empty, the tiles of that wave run as K parts (work units of their
own); each part writes its FP32 partial tile to scratch and the part that
finishes last adds all parts in part order.  These tests check that the plan
really splits at the chosen shapes, that integer products stay bit-exact
(every partial sum is an exact integer), that uniform inputs stay within the
split path's tolerance against the oracle, and that the result does not
depend on which part finishes last (two calls agree bit for bit).
"""
import numpy as np
import pytest
import torch

import synth
from gpu_util import assert_full, dev, run_gemm, run_packed, sampled_check

pytestmark = pytest.mark.gpu

# (n, m, p): every tile split (fewer tiles than SMs); whole tiles plus a split
# last wave (more tiles than SMs); one tile split many ways (skinny).  m >= 2237
# keeps the first two on the two-part (three-product) kind.
ALL_SPLIT = (1000, 3000, 1000)
MIXED = (5120, 2304, 1024)
ONE_TILE = (129, 4096, 70)


def _plan(mm, shape):
    st, tiles, split_from, split_s = mm.mm_tune_query_tail(*shape)
    assert st == mm.MM_OK
    return tiles, split_from, split_s


def test_plan_splits_the_tail(mmlib):
    tiles, f, s = _plan(mmlib, ALL_SPLIT)
    assert s > 1 and f == 0 and tiles > 0
    tiles, f, s = _plan(mmlib, MIXED)
    assert s > 1 and 0 < f < tiles
    tiles, f, s = _plan(mmlib, ONE_TILE)
    assert tiles == 2 and s > 1
    # a product whose tiles fill whole waves is not split
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    _, bn, _, _, _ = mmlib.mm_tune_query(128 * n_sm, 4096, 256)
    if bn == 256:
        tiles, f, s = _plan(mmlib, (128 * n_sm, 4096, 256))
        assert tiles == n_sm and s == 1 and f == tiles


@pytest.mark.parametrize("shape", [ALL_SPLIT, MIXED, ONE_TILE],
                         ids=["all_split", "mixed", "one_tile"])
def test_tail_small_integers_bit_exact(mmlib, shape):
    """Entries in [-8, 8]: every partial tile and their sum are exact integers
    below 2^24, so the split product equals the exact product bit for bit."""
    n, m, p = shape
    A = synth.small_ints(2101, (n, m))
    B = synth.small_ints(2102, (m, p))
    C = run_packed(mmlib, A, B, mmlib.MM_MODE_SPLIT_BF16X3)
    exact = A.astype(np.float64) @ B.astype(np.float64)  # exact: |c| < 2^53
    assert np.array_equal(C.astype(np.float64), exact)


@pytest.mark.parametrize("shape", [ALL_SPLIT, ONE_TILE], ids=["all_split", "one_tile"])
def test_tail_uniform_full_oracle(mmlib, shape):
    n, m, p = shape
    A = synth.uniform_pm1(2201, (n, m))
    B = synth.uniform_pm1(2202, (m, p))
    C = run_packed(mmlib, A, B, mmlib.MM_MODE_SPLIT_BF16X3)
    assert_full(C, A, B, "f32")


def test_tail_uniform_mixed_sampled(mmlib):
    n, m, p = MIXED
    A = synth.uniform_pm1(2301, (n, m))
    B = synth.uniform_pm1(2302, (m, p))
    C = run_packed(mmlib, A, B, mmlib.MM_MODE_SPLIT_BF16X3)
    sampled_check(C, A, B, "f32")


def test_tail_deterministic_and_batch_invariant(mmlib):
    """Two calls give the same bits whichever part of a split tile finishes
    last, and a grouped call holding the product beside another one gives
    the same bits again: the split is a property of the product's shape, not
    of the launch it runs in."""
    mm = mmlib
    n, m, p = MIXED
    A = synth.uniform_pm1(2401, (n, m))
    B = synth.uniform_pm1(2402, (m, p))
    dA, dB = dev(A), dev(B)
    outs = []
    for _ in range(2):
        C = torch.full((n, p), float("nan"), device="cuda")
        assert mm.mm_gemm_grouped([(n, m, p, dA, dB, C)], mm.MM_F32, mm.MM_MODE_SPLIT_BF16X3) == 0
        outs.append(C.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    for other in ((64, m, 64), (300, 700, 200)):  # same split kind / another kind
        Cg = torch.full((n, p), float("nan"), device="cuda")
        a = torch.zeros(other[0] * other[1], device="cuda")
        b = torch.zeros(other[1] * other[2], device="cuda")
        c = torch.zeros(other[0] * other[2], device="cuda")
        st = mm.mm_gemm_grouped([(n, m, p, dA, dB, Cg), other + (a, b, c)], mm.MM_F32,
                                mm.MM_MODE_SPLIT_BF16X3)
        assert st == 0
        assert np.array_equal(Cg.cpu().numpy(), outs[0])


def test_tail_three_part_kind(mmlib):
    """m = 2100 (< 2237) takes the three-part split (six products); with 320
    tiles the last wave is split too.  Integer inputs stay exact; uniform
    inputs stay within the tolerance on sampled entries and Freivalds."""
    n, m, p = 5000, 2100, 1024
    tiles, f, s = _plan(mmlib, (n, m, p))
    assert s > 1 and 0 < f < tiles
    A = synth.small_ints(2501, (n, m))
    B = synth.small_ints(2502, (m, p))
    C = run_packed(mmlib, A, B, mmlib.MM_MODE_SPLIT_BF16X3)
    assert np.array_equal(C.astype(np.float64), A.astype(np.float64) @ B.astype(np.float64))
    A = synth.uniform_pm1(2503, (n, m))
    B = synth.uniform_pm1(2504, (m, p))
    C = run_packed(mmlib, A, B, mmlib.MM_MODE_SPLIT_BF16X3)
    sampled_check(C, A, B, "f32")


def test_tail_fp8_small_integers(mmlib):
    """The e4m3 path plans its tail from its own K blocks (128 values per pack
    row); at 5120 x 8192 x 1024 (160 tiles of 128 x 256, 64 K blocks) its last
    wave is split.  Small integers are exact through e4m3 and through the
    ordered sum of the parts (|c| <= 8192 * 64 < 2^24)."""
    n, m, p = 5120, 8192, 1024
    A = synth.small_ints(2601, (n, m))
    B = synth.small_ints(2602, (m, p))
    C = run_gemm(mmlib, A, B, mmlib.MM_MODE_FP8)
    assert np.array_equal(C.astype(np.float64), A.astype(np.float64) @ B.astype(np.float64))


def test_tail_with_scaled_operands(mmlib):
    """Rows of A at 2^-70 / 2^60 and columns of B at 2^-45 / 2^45 (outside
    the range packed unscaled, and every product still a normal FP32 number)
    force the re-pack of both operands with power-of-two scales; the split
    tiles' parts are summed unscaled and the row and column scales applied
    once to the sum.  Every tile is split here (1000 x 3000 x 1000), and the
    full oracle checks every entry."""
    n, m, p = ALL_SPLIT
    ea = synth.row_scale_exponents(2701, n, choices=(-70, 60))
    eb = synth.row_scale_exponents(2702, p, choices=(-45, 45))
    A = (synth.uniform_pm1(2703, (n, m)).astype(np.float64) * np.ldexp(1.0, ea)[:, None]).astype(np.float32)
    B = (synth.uniform_pm1(2704, (m, p)).astype(np.float64) * np.ldexp(1.0, eb)[None, :]).astype(np.float32)
    C = run_packed(mmlib, A, B, mmlib.MM_MODE_SPLIT_BF16X3)
    assert np.all(np.isfinite(C))
    assert_full(C, A, B, "f32")
