"""C = alpha (A.B) + beta D with the epilogue fused into the product
(mm_gemm_axpby): the paper's matrix addition/subtraction (results section)
applied by the kernel that writes C.  For every path and every kernel that
writes C (SIMT one-pass and K-sliced, DGEMM, the split path's packed kernel
with and without its tail split and its fused split-K kernel, the three-part
kind, FP8's uniform and blockwise tiles, the FP64 emulation and its gate's
fallback), against mm_gemm's own product x of the same inputs:
  alpha = 1, beta = 0 gives x bit for bit; alpha = 2, beta = 0 gives 2x;
  alpha = 1, beta = -1 gives x - d correctly rounded (the host's IEEE result);
  general coefficients give fma(alpha, x, beta d) within an ulp;
  D = C (in place) gives the same bits as a separate D;
  the epilogue adds no kernel launch, except on FP8, which runs it as a pass
  of its own and adds exactly one;
and against the oracle's alpha (A.B) + beta D within the product's tolerance
plus the epilogue's roundings."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import dev
from oracle import ozaki

pytestmark = pytest.mark.gpu

# (name, mode, f64, (n, m, p)); the kernel that writes C in the comment
CASES = [
    ("simt_onepass", "SIMT", False, (1280, 256, 1024)),       # 128x128 tiles, vector stores
    ("simt_onepass_ragged", "SIMT", False, (1290, 100, 1030)),  # edge stores
    ("simt_slices", "SIMT", False, (200, 2048, 150)),         # K slices + fixed-order sum
    ("simt_one_slice", "SIMT", False, (70, 100, 33)),         # one slice writes C
    ("dgemm_onepass", "DGEMM", True, (640, 128, 650)),
    ("dgemm_slices", "DGEMM", True, (64, 4096, 64)),
    ("split_packed", "SPLIT_BF16X3", False, (2048, 512, 2048)),  # tc_gemm plain stores
    ("split_tail", "SPLIT_BF16X3", False, (5120, 2304, 1024)),   # tc_gemm, split last wave
    ("split_fused", "SPLIT_BF16X3", False, (1000, 3000, 1000)),  # fused split-K kernel
    ("split_fused_skinny", "SPLIT_BF16X3", False, (129, 4096, 70)),
    ("split_x6", "SPLIT_BF16X6", False, (1536, 512, 1536)),
    ("fp8", "FP8", False, (1024, 1024, 1024)),
    ("ozaki", "OZAKI", True, (300, 517, 260)),
]


def _inputs(name, n, m, p, f64):
    seed = sum(map(ord, name))
    if f64:
        A = synth.uniform_pm1_f64(seed, (n, m))
        B = synth.uniform_pm1_f64(seed + 1, (m, p))
        D = synth.uniform_pm1_f64(seed + 2, (n, p)) * 8.0
    else:
        A = synth.uniform_pm1(seed, (n, m))
        B = synth.uniform_pm1(seed + 1, (m, p))
        D = synth.uniform_pm1(seed + 2, (n, p)) * np.float32(8.0)
        if name == "fp8":
            # row tile 0 of A with one K block 2^12 larger: its tiles take the
            # blockwise kernel, the others the uniform one
            A[:128, 128:256] *= np.float32(2.0 ** 12)
    return A, B, D


def _gemm(mm, n, m, p, dA, dB, f64, mode):
    tdt = torch.float64 if f64 else torch.float32
    C = torch.full((n, p), float("nan"), dtype=tdt, device="cuda")
    st = mm.mm_gemm(n, m, p, dA, dB, C, mm.MM_F64 if f64 else mm.MM_F32, mode)
    assert st == mm.MM_OK, mm.mm_strerror(st)
    return C


def _axpby(mm, n, m, p, alpha, dA, dB, beta, dD, f64, mode, C=None):
    tdt = torch.float64 if f64 else torch.float32
    if C is None:
        C = torch.full((n, p), float("nan"), dtype=tdt, device="cuda")
    st = mm.mm_gemm_axpby(n, m, p, alpha, dA, dB, beta, dD, C,
                          mm.MM_F64 if f64 else mm.MM_F32, mode)
    assert st == mm.MM_OK, mm.mm_strerror(st)
    return C


def _same(C, ref):
    C, ref = np.asarray(C), np.asarray(ref)
    bad = np.count_nonzero(C != ref)
    assert bad == 0, "%d of %d entries differ" % (bad, C.size)


@pytest.fixture
def gate_on(mmlib):
    assert mmlib.mm_ozaki_gate(1) == mmlib.MM_OK
    assert mmlib.mm_ozaki_slices(ozaki.DEFAULT_SLICES) == mmlib.MM_OK
    yield mmlib


@pytest.mark.parametrize("name,mode,f64,shape", CASES, ids=[c[0] for c in CASES])
def test_epilogue_against_the_product(gate_on, name, mode, f64, shape):
    mm = gate_on
    md = getattr(mm, "MM_MODE_" + mode)
    n, m, p = shape
    A, B, D = _inputs(name, n, m, p, f64)
    tdt = torch.float64 if f64 else torch.float32
    dA, dB, dD = dev(A, tdt), dev(B, tdt), dev(D, tdt)
    x = _gemm(mm, n, m, p, dA, dB, f64, md).cpu().numpy()
    dt = np.float64 if f64 else np.float32
    _same(_axpby(mm, n, m, p, 1.0, dA, dB, 0.0, None, f64, md).cpu().numpy(), x)
    _same(_axpby(mm, n, m, p, 2.0, dA, dB, 0.0, None, f64, md).cpu().numpy(), dt(2) * x)
    sub = _axpby(mm, n, m, p, 1.0, dA, dB, -1.0, dD, f64, md).cpu().numpy()
    _same(sub, x - D)
    # in place: C holds D on entry
    Cin = dD.clone()
    _same(_axpby(mm, n, m, p, 1.0, dA, dB, -1.0, Cin, f64, md, C=Cin).cpu().numpy(), sub)
    # general coefficients: fma(alpha, x, fl(beta d)), one rounding of the sum
    alpha, beta = 0.75, -1.5
    got = _axpby(mm, n, m, p, alpha, dA, dB, beta, dD, f64, md).cpu().numpy()
    t = dt(beta) * D  # fl(beta d) in the element type, as the kernels round it
    if not f64:
        # alpha x (26 significant bits) and t (24) on grids and magnitudes
        # that keep their sum exact in FP64: one rounding to FP32 remains
        want = alpha * x.astype(np.float64) + t.astype(np.float64)
        ulp = np.spacing(np.abs(want).astype(np.float32)).astype(np.float64)
        assert np.all(np.abs(got.astype(np.float64) - want) <= ulp), name
    else:
        # FP64: within two roundings of the magnitudes summed
        want = alpha * x + t
        assert np.all(np.abs(got - want) <= 2.0 ** -52 * (np.abs(alpha * x) + np.abs(t))), name


ORACLE_CASES = [c for c in CASES if c[1] != "FP8" and c[3][0] * c[3][1] * c[3][2] <= 2 ** 31]


@pytest.mark.parametrize("name,mode,f64,shape", ORACLE_CASES, ids=[c[0] for c in ORACLE_CASES])
def test_epilogue_against_the_oracle(gate_on, name, mode, f64, shape):
    """The result against the oracle's alpha (A.B) + beta D, with the error
    normalised by |alpha| (|A|.|B|) + |beta| |D|: within the path's product
    tolerance plus three roundings of the element type (beta d, the fma, and
    the product's own magnitude)."""
    mm = gate_on
    md = getattr(mm, "MM_MODE_" + mode)
    n, m, p = shape
    A, B, D = _inputs(name, n, m, p, f64)
    tdt = torch.float64 if f64 else torch.float32
    C = _axpby(mm, n, m, p, -0.3, dev(A, tdt), dev(B, tdt), 1.7, dev(D, tdt), f64, md).cpu().numpy()
    ref, norm = oracle.default().axpby(-0.3, A, B, 1.7, D)
    u = 2.0 ** -53 if f64 else 2.0 ** -24
    tol = oracle.tolerance(m, "f64" if f64 else "f32") + 3 * u
    e = oracle.rel_errors(C, ref, norm)
    assert e.max() <= tol, "max e %g > %g" % (e.max(), tol)


LAUNCH_CASES = [c for c in CASES if c[0] in (
    "simt_onepass", "simt_slices", "dgemm_slices", "split_packed", "split_tail", "split_fused",
    "split_fused_skinny", "fp8", "ozaki")]


@pytest.mark.parametrize("name,mode,f64,shape", LAUNCH_CASES, ids=[c[0] for c in LAUNCH_CASES])
def test_epilogue_launches(gate_on, name, mode, f64, shape):
    mm = gate_on
    md = getattr(mm, "MM_MODE_" + mode)
    n, m, p = shape
    A, B, D = _inputs(name, n, m, p, f64)
    tdt = torch.float64 if f64 else torch.float32
    dA, dB, dD = dev(A, tdt), dev(B, tdt), dev(D, tdt)
    C = torch.empty((n, p), dtype=tdt, device="cuda")
    dt = mm.MM_F64 if f64 else mm.MM_F32

    def count(fn):
        fn()
        torch.cuda.synchronize()
        l0 = mm.mm_launch_count()
        assert fn() == mm.MM_OK
        torch.cuda.synchronize()
        return mm.mm_launch_count() - l0

    plain = count(lambda: mm.mm_gemm(n, m, p, dA, dB, C, dt, md))
    fused = count(lambda: mm.mm_gemm_axpby(n, m, p, 0.5, dA, dB, -1.0, dD, C, dt, md))
    assert fused == plain + (1 if mode == "FP8" else 0), (plain, fused)


def test_gate_fallback_in_place(gate_on):
    """Entries spread over 2^-40 .. 2^40: the FP64 emulation's gate fails and
    the FP64 FMA product writes C.  In place (D = C) the fallback still reads
    the original D: the result is the DGEMM mode's, bit for bit."""
    mm = gate_on

    def wide(seed, shape):
        return (synth.uniform_pm1_f64(seed, shape) *
                synth.pow2_int(seed + 1, shape, -40, 40).astype(np.float64))

    n, m, p = 129, 300, 70
    A, B = wide(7100, (n, m)), wide(7102, (m, p))
    D = synth.uniform_pm1_f64(7104, (n, p))
    dA, dB = dev(A, torch.float64), dev(B, torch.float64)
    res = []
    for md in (mm.MM_MODE_OZAKI, mm.MM_MODE_DGEMM):
        C = dev(D, torch.float64)
        res.append(_axpby(mm, n, m, p, 1.0, dA, dB, 1.0, C, True, md, C=C).cpu().numpy())
    _same(res[0], res[1])
    C = _axpby(mm, n, m, p, 1.0, dA, dB, 1.0, dev(D, torch.float64), True,
               mm.MM_MODE_OZAKI).cpu().numpy()
    _same(C, res[1])


@pytest.mark.parametrize("f64", [False, True])
def test_no_product_terms(mmlib, f64):
    """alpha = 0 or m = 0: C = beta D exactly, A and B not read (NULL here);
    beta = 0 as well: C = 0 without reading D; beta = 0 with the product: a
    NaN in D does not reach C."""
    mm = mmlib
    tdt = torch.float64 if f64 else torch.float32
    dt = mm.MM_F64 if f64 else mm.MM_F32
    n, p = 33, 47
    D = synth.uniform_pm1(7200, (n, p)).astype(np.float64 if f64 else np.float32)
    dD = dev(D, tdt)
    for md in (mm.MM_MODE_AUTO,):
        C = torch.full((n, p), float("nan"), dtype=tdt, device="cuda")
        assert mm.mm_gemm_axpby(n, 10, p, 0.0, None, None, -3.0, dD, C, dt, md) == mm.MM_OK
        _same(C.cpu().numpy(), D * (np.float64(-3.0) if f64 else np.float32(-3.0)))
        C.fill_(float("nan"))
        assert mm.mm_gemm_axpby(n, 0, p, 1.0, None, None, 0.5, dD, C, dt, md) == mm.MM_OK
        _same(C.cpu().numpy(), D * (np.float64(0.5) if f64 else np.float32(0.5)))
        C.fill_(float("nan"))
        assert mm.mm_gemm_axpby(n, 10, p, 0.0, None, None, 0.0, None, C, dt, md) == mm.MM_OK
        assert torch.all(C == 0)
    A = dev(synth.uniform_pm1(7202, (n, 64)), tdt)
    B = dev(synth.uniform_pm1(7203, (64, p)), tdt)
    Dn = torch.full((n, p), float("nan"), dtype=tdt, device="cuda")
    C = torch.empty((n, p), dtype=tdt, device="cuda")
    md = mm.MM_MODE_DGEMM if f64 else mm.MM_MODE_SPLIT_BF16X3
    assert mm.mm_gemm_axpby(n, 64, p, 1.0, A, B, 0.0, Dn, C, dt, md) == mm.MM_OK
    assert torch.isfinite(C).all()


def test_arguments(mmlib):
    mm = mmlib
    x = torch.zeros(64, device="cuda")
    host = np.zeros(64, np.float32)
    F32, SPLIT = mm.MM_F32, mm.MM_MODE_SPLIT_BF16X3
    assert mm.mm_gemm_axpby(8, 8, 8, 1.0, x, x, 1.0, None, x, F32, SPLIT) == mm.MM_EINVAL
    assert mm.mm_gemm_axpby_async(8, 8, 8, 1.0, x, x, 1.0, host, x, F32, SPLIT) == mm.MM_EINVAL
    C = torch.zeros(128, device="cuda")
    # D overlapping C without being C
    assert mm.mm_gemm_axpby(8, 8, 8, 1.0, x, x, 1.0, C[4:], C, F32, SPLIT) == mm.MM_EINVAL
    assert mm.mm_gemm_axpby(-1, 8, 8, 1.0, x, x, 0.0, None, x, F32, SPLIT) == mm.MM_EINVAL
    assert mm.mm_gemm_axpby(8, 8, 8, 1.0, x, x, 0.0, None, x, F32,
                            mm.MM_MODE_DGEMM) == mm.MM_EUNSUPPORTED
    assert mm.mm_gemm_axpby(0, 8, 8, 1.0, None, None, 1.0, None, None, F32, SPLIT) == mm.MM_OK
    assert mm.mm_gemm_axpby(8, 8, 8, 1.0, None, x, 0.0, None, x, F32, SPLIT) == mm.MM_EINVAL


@pytest.mark.parametrize("mode", ["SPLIT_BF16X3", "SIMT"])
def test_host_operands(mmlib, mode):
    """Host A, B, D and C (staged through library buffers) give the device
    call's bits, separate and in place (D = C on the host)."""
    mm = mmlib
    md = getattr(mm, "MM_MODE_" + mode)
    n, m, p = 300, 700, 260
    A = synth.uniform_pm1(7400, (n, m))
    B = synth.uniform_pm1(7401, (m, p))
    D = synth.uniform_pm1(7402, (n, p))
    want = _axpby(mm, n, m, p, 0.5, dev(A), dev(B), -2.0, dev(D), False, md).cpu().numpy()
    C = np.full((n, p), np.nan, np.float32)
    assert mm.mm_gemm_axpby(n, m, p, 0.5, A, B, -2.0, D, C, mm.MM_F32, md) == mm.MM_OK
    _same(C, want)
    C = D.copy()
    assert mm.mm_gemm_axpby(n, m, p, 0.5, A, B, -2.0, C, C, mm.MM_F32, md) == mm.MM_OK
    _same(C, want)
    # device A and B, host D and C
    C = np.full((n, p), np.nan, np.float32)
    assert mm.mm_gemm_axpby(n, m, p, 0.5, dev(A), dev(B), -2.0, D, C, mm.MM_F32, md) == mm.MM_OK
    _same(C, want)
    # host D overlapping host C without being C
    buf = np.zeros(2 * n * p, np.float32)
    Cv, Dv = buf[:n * p], buf[4:4 + n * p]
    assert mm.mm_gemm_axpby(n, m, p, 0.5, A, B, -2.0, Dv, Cv, mm.MM_F32, md) == mm.MM_EINVAL


def test_async_on_a_stream(mmlib):
    """The asynchronous form on a caller's stream gives the synchronous
    form's bits."""
    mm = mmlib
    n, m, p = 300, 700, 260
    dA = dev(synth.uniform_pm1(7300, (n, m)))
    dB = dev(synth.uniform_pm1(7301, (m, p)))
    dD = dev(synth.uniform_pm1(7302, (n, p)))
    C1 = _axpby(mm, n, m, p, 0.5, dA, dB, 2.0, dD, False, mm.MM_MODE_SPLIT_BF16X3)
    s = torch.cuda.Stream()
    C2 = torch.full((n, p), float("nan"), device="cuda")
    torch.cuda.synchronize()
    assert mm.mm_gemm_axpby_async(n, m, p, 0.5, dA, dB, 2.0, dD, C2, mm.MM_F32,
                                  mm.MM_MODE_SPLIT_BF16X3, s.cuda_stream) == mm.MM_OK
    s.synchronize()
    assert torch.equal(C1, C2)
