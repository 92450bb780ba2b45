"""The fused split-K kernel (mm_gemm's split path for products with few output
tiles): its plan, parity with the CPU oracle element by element on shapes
that exercise every reduction form (one CTA per tile, a cluster per tile, and
several clusters per tile meeting in global memory), ragged edges, unaligned
operands, the per-block power-of-two scaling, non-finite entries, exact
integer products, and determinism."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import assert_full, dev, fused_slices, run_gemm, sampled_check

pytestmark = pytest.mark.gpu

# (n, m, p) chosen to reach: S = 1 (tiny K), one cluster per tile (Q = 1,
# cluster of 2..8), several clusters per tile (Q > 1: the skinny products),
# ragged n, K blocks cut short (m not a multiple of 64), m below 64, and p
# below and above one 128-wide tile.  The kernel reads A and B with TMA, so
# m and p are multiples of 4 (other products take the packed path).
SHAPES = [(1, 4, 4), (3, 8, 12), (1000, 36, 32), (129, 68, 260), (300, 2300, 200),
          (64, 16384, 64), (130, 9000, 132), (7, 4100, 516), (257, 1024, 132),
          (128, 640, 128), (512, 512, 512)]


def _plan(mm, n, m, p):
    st, tiles, s, q, cs = mm.mm_tune_query_splitk(n, m, p)
    assert st == mm.MM_OK
    return tiles, s, q, cs


def test_plan(mmlib):
    mm = mmlib
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    tiles, s, q, cs = _plan(mm, 64, 16384, 64)
    assert tiles == 1 and s >= 64 and q > 1 and cs in (2, 4, 8) and s == q * cs
    tiles, s, q, cs = _plan(mm, 512, 512, 512)
    assert tiles == 16 and s >= 2 and tiles * s <= n_sm
    # 1024^3: eight K blocks per slice; 1024 x 2048 x 1024 would need sixteen
    # and takes the packed path
    assert _plan(mm, 1024, 1024, 1024)[1] >= 2
    assert _plan(mm, 1024, 2048, 1024)[1] == 0
    tiles, s, q, cs = _plan(mm, 3, 8, 12)
    assert tiles == 1 and s == 1 and q == 1 and cs == 1
    # products that fill half the SMs with whole tiles keep the packed path
    assert _plan(mm, 8192, 8192, 8192)[1] == 0
    assert _plan(mm, 128 * n_sm, 512, 128)[1] == 0
    for shape in SHAPES:
        tiles, s, q, cs = _plan(mm, *shape)
        assert s > 0, shape
        assert s == q * cs and cs in (1, 2, 4, 8)
        assert s <= (shape[1] + 63) // 64  # at least one K block per slice


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("mode", ["x3", "x6"])
def test_uniform_matches_oracle(mmlib, shape, mode):
    n, m, p = shape
    A = synth.uniform_pm1(3300 + n, (n, m))
    B = synth.uniform_pm1(3400 + p, (m, p))
    md = mmlib.MM_MODE_SPLIT_BF16X3 if mode == "x3" else mmlib.MM_MODE_SPLIT_BF16X6
    C = run_gemm(mmlib, A, B, md)
    assert_full(C, A, B, "f32")


@pytest.mark.parametrize("shape", [(64, 16384, 64), (300, 2300, 200), (129, 68, 260)],
                         ids=lambda s: "x".join(map(str, s)))
def test_small_integers_exact(mmlib, shape):
    """Entries in [-8, 8]: every block's partial product, every sum of blocks
    and of slices is an exact integer below 2^24."""
    n, m, p = shape
    A = synth.small_ints(3501, (n, m))
    B = synth.small_ints(3502, (m, p))
    C = run_gemm(mmlib, A, B, mmlib.MM_MODE_SPLIT_BF16X3)
    exact = A.astype(np.float64) @ B.astype(np.float64)
    assert np.array_equal(C.astype(np.float64), exact)


def test_deterministic(mmlib):
    """Several clusters of one tile meet in global memory, and whichever
    arrives last adds the others in cluster order: two calls agree bit for
    bit."""
    mm = mmlib
    n, m, p = 64, 16384, 64
    assert _plan(mm, n, m, p)[2] > 1
    A = dev(synth.uniform_pm1(3601, (n, m)))
    B = dev(synth.uniform_pm1(3602, (m, p)))
    outs = []
    for _ in range(3):
        C = torch.full((n, p), float("nan"), device="cuda")
        assert mm.mm_gemm(n, m, p, A, B, C, mm.MM_F32, mm.MM_MODE_SPLIT_BF16X3) == 0
        outs.append(C)
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])


def test_scaled_blocks(mmlib):
    """Rows of A at 2^-70 / 2^60 and columns of B at 2^-45 / 2^45 put entries
    outside [2^-40, 2^40] (every product still a normal FP32 number): those
    K blocks are split after per-row / per-column power-of-two scaling and
    unscaled exactly before the blocks are added.  The first row tile keeps
    ordinary rows; its blocks are still scaled where B is out of range.  Full
    oracle check; then rows at 2^-120 / 2^100 against a B in range."""
    n, m, p = 300, 1000, 200
    A0 = synth.uniform_pm1(3701, (n, m)).astype(np.float64)
    B0 = synth.uniform_pm1(3702, (m, p)).astype(np.float64)
    A, B = A0, B0
    ea = synth.row_scale_exponents(3703, n, choices=(-70, 60))
    ea[:128] = 0  # the first row tile stays in range
    eb = synth.row_scale_exponents(3704, p, choices=(-45, 45))
    A = (A * np.ldexp(1.0, ea)[:, None]).astype(np.float32)
    B = (B * np.ldexp(1.0, eb)[None, :]).astype(np.float32)
    for md in (mmlib.MM_MODE_SPLIT_BF16X3, mmlib.MM_MODE_SPLIT_BF16X6):
        C = run_gemm(mmlib, A, B, md)
        assert np.all(np.isfinite(C))
        assert_full(C, A, B, "f32")
    A = (A0 * np.ldexp(1.0, synth.row_scale_exponents(3705, n))[:, None]).astype(np.float32)
    B = B0.astype(np.float32)
    C = run_gemm(mmlib, A, B, mmlib.MM_MODE_SPLIT_BF16X3)
    assert np.all(np.isfinite(C))
    assert_full(C, A, B, "f32")


def test_pow2_exponent_stress(mmlib):
    """Entries s 2^e with e real in [-20, 20): every block in range (no
    scaling), products spread over 80 binades of |A||B|."""
    n, m, p = 200, 4096, 152
    A = synth.pow2_real(3801, (n, m))
    B = synth.pow2_real(3802, (m, p))
    C = run_gemm(mmlib, A, B, mmlib.MM_MODE_SPLIT_BF16X3)
    assert_full(C, A, B, "f32")


def test_nonfinite_row(mmlib):
    """A NaN in A makes its row of C non-finite (the block holding it is
    scaled with exponent 0 for that row, and the NaN propagates); the other
    rows stay within the tolerance."""
    n, m, p = 40, 500, 60
    A = synth.uniform_pm1(3901, (n, m))
    B = synth.uniform_pm1(3902, (m, p))
    A[3, 7] = np.nan
    C = run_gemm(mmlib, A, B, mmlib.MM_MODE_SPLIT_BF16X3)
    assert not np.isfinite(C[3]).any()
    keep = np.ones(n, bool)
    keep[3] = False
    assert np.isfinite(C[keep]).all()
    assert_full(C[keep], A[keep], B, "f32")


def test_guard_words(mmlib):
    """C is written exactly on its n x p entries: guard words around it stay."""
    mm = mmlib
    n, m, p = 67, 2132, 44
    A = synth.uniform_pm1(4001, (n, m))
    B = synth.uniform_pm1(4002, (m, p))
    assert fused_slices(mm, n, m, p) > 0
    bufC = torch.full((n * p + 64,), 7.0, device="cuda")
    st = mm.mm_gemm(n, m, p, dev(A), dev(B), bufC[32:32 + n * p], mm.MM_F32,
                    mm.MM_MODE_SPLIT_BF16X3)
    assert st == 0
    assert torch.all(bufC[:32] == 7.0) and torch.all(bufC[32 + n * p:] == 7.0)
    assert_full(bufC[32:32 + n * p].reshape(n, p).cpu().numpy(), A, B, "f32")


@pytest.mark.parametrize("case", ["offset", "odd_m", "odd_p"])
def test_unaligned_takes_packed_path(mmlib, case):
    """Operands the TMA loads cannot take (a start off a 16-byte boundary, or
    a row pitch that is not a multiple of 16 bytes) run on the packed path:
    the result equals a grouped call of the product bit for bit."""
    mm = mmlib
    n, m, p = 67, (2131 if case == "odd_m" else 2132), (45 if case == "odd_p" else 44)
    A = synth.uniform_pm1(4011, (n, m))
    B = synth.uniform_pm1(4012, (m, p))
    off = 1 if case == "offset" else 0
    bufA = torch.zeros(n * m + 1, device="cuda")
    bufB = torch.zeros(m * p + 1, device="cuda")
    bufA[off:off + n * m] = dev(A).reshape(-1)
    bufB[off:off + m * p] = dev(B).reshape(-1)
    dA, dB = bufA[off:off + n * m], bufB[off:off + m * p]
    C1 = torch.full((n, p), float("nan"), device="cuda")
    C2 = torch.full((n, p), float("nan"), device="cuda")
    assert mm.mm_gemm(n, m, p, dA, dB, C1, mm.MM_F32, mm.MM_MODE_SPLIT_BF16X3) == 0
    assert mm.mm_gemm_grouped([(n, m, p, dA, dB, C2)], mm.MM_F32, mm.MM_MODE_SPLIT_BF16X3) == 0
    assert torch.equal(C1, C2)
    assert_full(C1.cpu().numpy(), A, B, "f32")


def test_against_packed_path(mmlib):
    """The fused and the packed path (a grouped call of one product) agree
    within the tolerance on the same inputs."""
    mm = mmlib
    n, m, p = 300, 2300, 200
    assert fused_slices(mm, n, m, p) > 0
    A = synth.uniform_pm1(4101, (n, m))
    B = synth.uniform_pm1(4102, (m, p))
    dA, dB = dev(A), dev(B)
    C1 = torch.full((n, p), float("nan"), device="cuda")
    C2 = torch.full((n, p), float("nan"), device="cuda")
    assert mm.mm_gemm(n, m, p, dA, dB, C1, mm.MM_F32, mm.MM_MODE_SPLIT_BF16X3) == 0
    assert mm.mm_gemm_grouped([(n, m, p, dA, dB, C2)], mm.MM_F32, mm.MM_MODE_SPLIT_BF16X3) == 0
    absref = np.abs(A.astype(np.float64)) @ np.abs(B.astype(np.float64))
    e = oracle.rel_errors(C1.cpu().numpy(), C2.cpu().numpy().astype(np.float64), absref)
    assert e.max() <= oracle.tolerance(m, "f32")


def test_async_on_a_stream(mmlib):
    """Queued on a caller stream and synchronised: the same bits as the
    synchronous call."""
    mm = mmlib
    n, m, p = 64, 16384, 64
    A = dev(synth.uniform_pm1(4201, (n, m)))
    B = dev(synth.uniform_pm1(4202, (m, p)))
    C1 = torch.full((n, p), float("nan"), device="cuda")
    C2 = torch.full((n, p), float("nan"), device="cuda")
    assert mm.mm_gemm(n, m, p, A, B, C1, mm.MM_F32, mm.MM_MODE_SPLIT_BF16X3) == 0
    s = torch.cuda.Stream()
    for _ in range(5):
        assert mm.mm_gemm_async(n, m, p, A, B, C2, mm.MM_F32, mm.MM_MODE_SPLIT_BF16X3, s) == 0
    assert mm.mm_sync(s) == 0
    assert torch.equal(C1, C2)


def test_config3b_full_size(mmlib):
    """The skinny bandwidth-bound product of the stress workload at its full
    size, 64 x 16384 . 16384 x 64, against the full FP64 oracle, and its
    sampled / Freivalds check."""
    n, m, p = 64, 16384, 64
    A = synth.uniform_pm1(4301, (n, m))
    B = synth.uniform_pm1(4302, (m, p))
    C = run_gemm(mmlib, A, B, mmlib.MM_MODE_SPLIT_BF16X3)
    assert_full(C, A, B, "f32")
    sampled_check(C, A, B, "f32", count=1024, trials=1)
