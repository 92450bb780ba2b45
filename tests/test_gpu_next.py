"""The paper's related workloads: the complex product (Table 2's complex
float column), matrix addition/subtraction (results section) and the product
with a diagonal matrix (algorithms section), each against the oracle or an
exact closed form."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import dev

pytestmark = pytest.mark.gpu


def _cplx(seed, shape, ints=False):
    if ints:
        return (synth.small_ints(seed, shape) + 1j * synth.small_ints(seed + 1, shape)).astype(np.complex64)
    return (synth.uniform_pm1(seed, shape) + 1j * synth.uniform_pm1(seed + 1, shape)).astype(np.complex64)


def _run_cgemm(mm, A, B, mode):
    n, m = A.shape
    p = B.shape[1]
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    dC = torch.full((n, p), float("nan"), dtype=torch.complex64, device="cuda")
    st = mm.mm_cgemm(n, m, p, dA, dB, dC, mode)
    assert st == mm.MM_OK, mm.mm_strerror(st)
    return dC.cpu().numpy()


@pytest.mark.parametrize("shape", [(1, 1, 1), (37, 53, 29), (300, 200, 520), (129, 2300, 70)],
                         ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("mode", ["simt", "split"])
def test_cgemm_matches_oracle(mmlib, shape, mode):
    n, m, p = shape
    md = mmlib.MM_MODE_SIMT if mode == "simt" else mmlib.MM_MODE_SPLIT_BF16X3
    A = _cplx(1400, (n, m))
    B = _cplx(1410, (m, p))
    C = _run_cgemm(mmlib, A, B, md)
    ref, absref = oracle.default().cgemm(A, B)
    e = oracle.rel_errors_complex(C, ref, absref)
    assert e.max() <= oracle.tolerance(m, "c32"), e.max()


@pytest.mark.parametrize("mode", ["simt", "split"])
def test_cgemm_small_integers_exact(mmlib, mode):
    md = mmlib.MM_MODE_SIMT if mode == "simt" else mmlib.MM_MODE_SPLIT_BF16X3
    A = _cplx(1420, (64, 300), ints=True)
    B = _cplx(1430, (300, 96), ints=True)
    C = _run_cgemm(mmlib, A, B, md)
    exact = A.astype(np.complex128) @ B.astype(np.complex128)
    assert np.array_equal(C.astype(np.complex128), exact)


def test_cgemm_args(mmlib):
    mm = mmlib
    x = torch.zeros(8, dtype=torch.complex64, device="cuda")
    assert mm.mm_cgemm(2, 2, 2, x, x, x, mm.MM_MODE_DGEMM) == mm.MM_EUNSUPPORTED
    assert mm.mm_cgemm(-1, 2, 2, x, x, x, mm.MM_MODE_SIMT) == mm.MM_EINVAL
    assert mm.mm_cgemm(0, 2, 2, None, None, None, mm.MM_MODE_SIMT) == mm.MM_OK
    C = torch.full((2, 3), 1 + 1j, dtype=torch.complex64, device="cuda")
    assert mm.mm_cgemm(2, 0, 3, x, x, C, mm.MM_MODE_AUTO) == mm.MM_OK
    assert torch.all(C == 0)


@pytest.mark.parametrize("f64", [False, True])
@pytest.mark.parametrize("shape", [(4096, 4096), (33, 7), (1, 1)], ids=lambda s: "x".join(map(str, s)))
def test_add_sub_exact(mmlib, f64, shape):
    """alpha = 1, beta = +-1: one correctly rounded addition or subtraction per
    entry, bit for bit the host's IEEE result."""
    n, p = shape
    dt = np.float64 if f64 else np.float32
    A = synth.uniform_pm1(1500, (n, p)).astype(dt)
    B = synth.uniform_pm1(1501, (n, p)).astype(dt)
    tdt = torch.float64 if f64 else torch.float32
    for beta in (1.0, -1.0):
        C = torch.full((n, p), float("nan"), dtype=tdt, device="cuda")
        st = mmlib.mm_add(n, p, 1.0, dev(A), beta, dev(B), C,
                          mmlib.MM_F64 if f64 else mmlib.MM_F32)
        assert st == 0
        assert np.array_equal(C.cpu().numpy(), A + dt(beta) * B)


def test_add_general_coefficients(mmlib):
    n, p = 257, 129
    A = synth.uniform_pm1(1510, (n, p))
    B = synth.uniform_pm1(1511, (n, p))
    C = torch.zeros((n, p), device="cuda")
    assert mmlib.mm_add(n, p, 0.75, dev(A), -2.5, dev(B), C, mmlib.MM_F32) == 0
    ref = 0.75 * A.astype(np.float64) - 2.5 * B.astype(np.float64)
    bound = 2.0 ** -23 * (np.abs(0.75 * A) + np.abs(2.5 * B)).astype(np.float64)
    assert np.all(np.abs(C.cpu().numpy() - ref) <= bound)


@pytest.mark.parametrize("f64", [False, True])
@pytest.mark.parametrize("side", [0, 1])
@pytest.mark.parametrize("shape", [(300, 520), (2500, 2052), (37, 4)],
                         ids=lambda s: "x".join(map(str, s)))
def test_diag_exact(mmlib, f64, side, shape):
    """c_ij = x_ij d_j (side 0) or d_i x_ij (side 1): one correctly rounded
    product per entry; agrees with the dense product through the general path
    on the same matrices.  2500 x 2052 has more 16-byte vectors than four
    strides of the persistent grid and a row length (513 vectors) that does
    not divide the stride, so the unrolled loop, its row wrap and the tail
    loop all run."""
    n, p = shape
    dt = np.float64 if f64 else np.float32
    X = synth.uniform_pm1(1520, (n, p)).astype(dt)
    d = synth.uniform_pm1(1521, p if side == 0 else n).astype(dt)
    tdt = torch.float64 if f64 else torch.float32
    C = torch.full((n, p), float("nan"), dtype=tdt, device="cuda")
    st = mmlib.mm_diag(n, p, dev(X), dev(d), C, side, mmlib.MM_F64 if f64 else mmlib.MM_F32)
    assert st == 0
    exact = X * d[None, :] if side == 0 else d[:, None] * X
    assert np.array_equal(C.cpu().numpy(), exact)
    if n * p > 10 ** 6:
        return  # the dense oracle product is too slow at this size; the exact check stands
    ref = oracle.default().gemm(X, np.diag(d)) if side == 0 else oracle.default().gemm(np.diag(d), X)
    assert np.array_equal(C.cpu().numpy().astype(np.float64), ref.astype(dt).astype(np.float64))


def test_diag_add_args(mmlib):
    mm = mmlib
    x = torch.zeros(4, device="cuda")
    assert mm.mm_diag(2, 2, x, x, x, 2, mm.MM_F32) == mm.MM_EINVAL
    assert mm.mm_add(2, 2, 1.0, np.zeros(4, np.float32), 1.0, x, x, mm.MM_F32) == mm.MM_EINVAL
    assert mm.mm_add(0, 5, 1.0, None, 1.0, None, None, mm.MM_F32) == mm.MM_OK


def test_add_diag_async_on_a_stream(mmlib):
    """The asynchronous forms on a caller stream give the same bits as the
    synchronous calls once the stream has been synchronised."""
    mm = mmlib
    n, p = 1000, 1028
    A = dev(synth.uniform_pm1(1530, (n, p)))
    B = dev(synth.uniform_pm1(1531, (n, p)))
    d = dev(synth.uniform_pm1(1532, p))
    s = torch.cuda.Stream()
    for side in (0, 1):
        dd = d if side == 0 else dev(synth.uniform_pm1(1533, n))
        C1 = torch.full((n, p), float("nan"), device="cuda")
        C2 = torch.full((n, p), float("nan"), device="cuda")
        assert mm.mm_diag(n, p, A, dd, C1, side, mm.MM_F32) == 0
        torch.cuda.synchronize()
        assert mm.mm_diag_async(n, p, A, dd, C2, side, mm.MM_F32, s) == 0
        assert mm.mm_sync(s) == 0
        assert torch.equal(C1, C2)
    C1 = torch.full((n, p), float("nan"), device="cuda")
    C2 = torch.full((n, p), float("nan"), device="cuda")
    assert mm.mm_add(n, p, 0.5, A, -3.0, B, C1, mm.MM_F32) == 0
    torch.cuda.synchronize()
    assert mm.mm_add_async(n, p, 0.5, A, -3.0, B, C2, mm.MM_F32, s) == 0
    assert mm.mm_sync(s) == 0
    assert torch.equal(C1, C2)
    x = torch.zeros(4, device="cuda")
    assert mm.mm_add_async(2, 2, 1.0, np.zeros(4, np.float32), 1.0, x, x, mm.MM_F32, s) == mm.MM_EINVAL
    assert mm.mm_diag_async(2, 2, x, x, x, 2, mm.MM_F32, s) == mm.MM_EINVAL
    assert mm.mm_add_async(0, 5, 1.0, None, 1.0, None, None, mm.MM_F32, s) == mm.MM_OK
