"""MM_MODE_OZAKI (FP64 emulated by the Ozaki scheme on the e4m3 tensor cores)
through the C ABI: with the accuracy gate off, equal bit for bit to the Ozaki
oracle (oracle/ozaki.py) on the same seeded inputs, at sizes that span several
tiles, ragged edges and several K chunks, for several slice counts; exact on
integers; within the FP64 tolerance of the exact product at 4096^3 (sampled
entries against Dot2 plus Freivalds); grouped, served and host-operand calls
give the same bits as a single device call; edge cases and argument checks.
With the gate on: products the method's error bound clears keep the
emulation's bits, and products it does not (magnitudes spread over many
binades, where the emulation itself misses the FP64 tolerance) are the FP64
FMA product's bits and meet the tolerance."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import dev, sampled_check
from oracle import ozaki

pytestmark = pytest.mark.gpu


@pytest.fixture
def mm(mmlib):
    """The library with the accuracy gate off (the bare method, comparable bit
    for bit with the oracle); slices and gate restored afterwards."""
    assert mmlib.mm_ozaki_gate(0) == mmlib.MM_OK
    yield mmlib
    assert mmlib.mm_ozaki_slices(ozaki.DEFAULT_SLICES) == mmlib.MM_OK
    assert mmlib.mm_ozaki_gate(1) == mmlib.MM_OK


def _run(mm, A, B, S=None, host=False, mode=None):
    if S is not None:
        assert mm.mm_ozaki_slices(S) == mm.MM_OK
    n, m = A.shape
    p = B.shape[1]
    if host:
        dA = torch.from_numpy(np.ascontiguousarray(A, np.float64))
        dB = torch.from_numpy(np.ascontiguousarray(B, np.float64))
        dC = torch.full((n, p), float("nan"), dtype=torch.float64)
    else:
        dA, dB = dev(A, torch.float64), dev(B, torch.float64)
        dC = torch.full((n, p), float("nan"), dtype=torch.float64, device="cuda")
    st = mm.mm_gemm(n, m, p, dA, dB, dC, mm.MM_F64, mm.MM_MODE_OZAKI if mode is None else mode)
    assert st == mm.MM_OK, mm.mm_strerror(st)
    return dC.cpu().numpy()


def _same(C, ref):
    assert C.shape == ref.shape
    assert np.array_equal(np.isnan(C), np.isnan(ref))
    ok = ~np.isnan(ref)
    bad = np.count_nonzero(C[ok] != ref[ok])
    assert bad == 0, "%d of %d entries differ (max |diff| %g)" % (
        bad, ok.sum(), np.max(np.abs(C[ok] - ref[ok])))


def _wide(seed, shape, lo=-40, hi=40):
    return synth.uniform_pm1_f64(seed, shape) * synth.pow2_int(seed + 1, shape, lo, hi).astype(np.float64)


@pytest.mark.parametrize("shape,S", [
    ((1, 1, 1), 12), ((64, 64, 64), 12), ((300, 517, 260), 12), ((257, 1000, 300), 2),
    ((257, 1000, 300), 8), ((129, 5500, 70), 12), ((130, 11000, 33), 6)])
def test_bit_exact_with_oracle(mm, shape, S):
    """Ragged shapes over several 128-row and 256-column tiles; (129, 5500, 70)
    with S = 12 and (130, 11000, 33) with S = 6 cross a K chunk boundary
    (chunks of 5376 and 10880 columns)."""
    n, m, p = shape
    A = synth.uniform_pm1_f64(4000 + n, (n, m))
    B = synth.uniform_pm1_f64(4001 + p, (m, p))
    _same(_run(mm, A, B, S), ozaki.gemm(A, B, S))


def test_bit_exact_wide_exponents(mm):
    A = _wide(4100, (257, 333))
    B = _wide(4102, (333, 129))
    A[5, :] = 0.0
    A[7, :] *= 2.0 ** -1000   # rows near the subnormal range
    B[:, 3] *= 2.0 ** 900
    for S in (4, 12):
        _same(_run(mm, A, B, S), ozaki.gemm(A, B, S))


def test_small_integers_exact(mm):
    A = synth.small_ints(4200, (129, 2000)).astype(np.float64)
    B = synth.small_ints(4201, (2000, 70)).astype(np.float64)
    C = _run(mm, A, B, 2)
    assert np.array_equal(C, (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64))


def test_fp64_tolerance_at_4096(mm):
    """The FP64 workload size: 4096 sampled entries against Dot2 and two
    Freivalds trials, elementwise tolerance 1e-14 sqrt(m)."""
    n = 4096
    A = synth.uniform_pm1_f64(4300, (n, n))
    B = synth.uniform_pm1_f64(4301, (n, n))
    C = _run(mm, A, B)
    emax, _ = sampled_check(C, A, B, "f64")
    assert emax < 1e-15


def test_edges(mm):
    A = synth.uniform_pm1_f64(4400, (150, 70))
    B = synth.uniform_pm1_f64(4401, (70, 90))
    A[2, :] = 0.0
    A[3, 11] = np.nan
    B[6, 40] = np.inf
    C = _run(mm, A, B)
    assert np.all(C[2, np.arange(90) != 40] == 0)
    assert np.all(np.isnan(C[3])) and np.all(np.isnan(C[:, 40]))
    _same(C, ozaki.gemm(A, B, ozaki.DEFAULT_SLICES))
    # m = 0 writes zeros; n = 0 is a no-op
    C0 = torch.full((4, 5), 7.0, dtype=torch.float64, device="cuda")
    e = torch.empty((4, 0), dtype=torch.float64, device="cuda")
    f = torch.empty((0, 5), dtype=torch.float64, device="cuda")
    assert mm.mm_gemm(4, 0, 5, e, f, C0, mm.MM_F64, mm.MM_MODE_OZAKI) == mm.MM_OK
    assert torch.all(C0 == 0)
    assert mm.mm_gemm(0, 3, 5, None, None, None, mm.MM_F64, mm.MM_MODE_OZAKI) == mm.MM_OK


def test_arguments(mm):
    assert mm.mm_ozaki_slices(1) == mm.MM_EINVAL
    assert mm.mm_ozaki_slices(13) == mm.MM_EINVAL
    assert mm.mm_ozaki_gate(2) == mm.MM_EINVAL
    assert mm.mm_ozaki_gate(-1) == mm.MM_EINVAL
    for S in (2, 12):
        assert mm.mm_ozaki_slices(S) == mm.MM_OK
    a = torch.zeros((8, 8), device="cuda")
    assert mm.mm_gemm(8, 8, 8, a, a, a, mm.MM_F32, mm.MM_MODE_OZAKI) == mm.MM_EUNSUPPORTED


def test_grouped_and_host_operands_match_single_calls(mm):
    shapes = [(200, 300, 100), (64, 5000, 64), (1, 7, 1)]
    mats = [(synth.uniform_pm1_f64(4500 + k, (n, m)), synth.uniform_pm1_f64(4510 + k, (m, p)))
            for k, (n, m, p) in enumerate(shapes)]
    single = [_run(mm, A, B) for A, B in mats]
    probs, outs = [], []
    for (n, m, p), (A, B) in zip(shapes, mats):
        C = torch.full((n, p), float("nan"), dtype=torch.float64, device="cuda")
        probs.append((n, m, p, dev(A, torch.float64), dev(B, torch.float64), C))
        outs.append(C)
    assert mm.mm_gemm_grouped(probs, mm.MM_F64, mm.MM_MODE_OZAKI) == mm.MM_OK
    for C, ref in zip(outs, single):
        _same(C.cpu().numpy(), ref)
    A, B = mats[0]
    _same(_run(mm, A, B, host=True), single[0])


def test_served_requests_match_single_calls(mmlib):
    mm = mmlib
    mm.mm_shutdown()
    assert mm.mm_init(device=0) == mm.MM_OK
    try:
        assert mm.mm_ozaki_slices(10) == mm.MM_OK
        assert mm.mm_ozaki_gate(0) == mm.MM_OK  # re-initialised: the gate is on again
        reqs = []
        for k, (n, m, p) in enumerate([(300, 200, 100), (128, 700, 256), (65, 65, 65)]):
            A = synth.uniform_pm1_f64(4600 + k, (n, m))
            B = synth.uniform_pm1_f64(4620 + k, (m, p))
            C = torch.full((n, p), float("nan"), dtype=torch.float64, device="cuda")
            dA, dB = dev(A, torch.float64), dev(B, torch.float64)
            st, rid = mm.mm_submit(n, m, p, dA, dB, C, mm.MM_F64, mm.MM_MODE_OZAKI)
            assert st == mm.MM_OK
            reqs.append((rid, A, B, C, dA, dB))
        for rid, A, B, C, _, _ in reqs:
            st, res, _, _ = mm.mm_wait(rid, 120.0)
            assert st == mm.MM_OK and res == mm.MM_OK
            _same(C.cpu().numpy(), ozaki.gemm(A, B, 10))
    finally:
        mm.mm_shutdown()
        assert mm.mm_init(device=0) == mm.MM_OK


def _exact(A, B):
    """Every entry of A.B by Dot2 (the oracle's compensated dot product) and
    the |A||B| normaliser."""
    n, p = A.shape[0], B.shape[1]
    I, J = np.meshgrid(np.arange(n), np.arange(p), indexing="ij")
    hi, lo, ab = oracle.default().entries(A, B, I.ravel(), J.ravel(), "dot2")
    return (hi + lo).reshape(n, p), ab.reshape(n, p)


def test_gate_keeps_emulation_where_the_bound_holds(mmlib):
    """Uniform entries: at S = 12 the bound clears every entry, so the gated
    product is the emulation's, bit for bit; at S = 8 it clears none at
    m = 1000 (the bound needs m of about 55 million there), so the gated product
    is the FP64 FMA product's."""
    mm = mmlib
    assert mm.mm_ozaki_gate(1) == mm.MM_OK
    try:
        A = synth.uniform_pm1_f64(7100, (257, 1000))
        B = synth.uniform_pm1_f64(7101, (1000, 300))
        _same(_run(mm, A, B, 12), ozaki.gemm(A, B, 12))
        _same(_run(mm, A, B, 8), _run(mm, A, B, mode=mm.MM_MODE_DGEMM))
    finally:
        assert mm.mm_ozaki_slices(ozaki.DEFAULT_SLICES) == mm.MM_OK


def test_gate_falls_back_where_the_emulation_misses(mmlib):
    """Entries spread over 2^-40 .. 2^40: the oracle's emulation at S = 12
    misses the FP64 tolerance on a share of the entries; the gated product is
    the FP64 FMA product, bit for bit, and meets the tolerance everywhere,
    including a row of NaN (NaN by design) and an all-zero row (zeros)."""
    mm = mmlib
    assert mm.mm_ozaki_gate(1) == mm.MM_OK
    try:
        A = _wide(7000, (129, 300))
        B = _wide(7002, (300, 70))
        A[4, :] = 0.0
        A[9, 17] = np.nan
        exact, ab = _exact(A, B)
        tol = oracle.tolerance(300, "f64")
        fin = np.isfinite(exact)
        emul = oracle.rel_errors(ozaki.gemm(A, B, 12)[fin], exact[fin], ab[fin])
        assert emul.max() > tol  # the bare method is not enough here
        C = _run(mm, A, B, 12)
        _same(C, _run(mm, A, B, mode=mm.MM_MODE_DGEMM))
        e = oracle.rel_errors(C[fin], exact[fin], ab[fin])
        assert e.max() <= tol, "max e %g > %g" % (e.max(), tol)
        assert np.all(np.isnan(C[9])) and np.all(C[4] == 0)
    finally:
        assert mm.mm_ozaki_slices(ozaki.DEFAULT_SLICES) == mm.MM_OK
