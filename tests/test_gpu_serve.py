"""Serving loop: continuous batching with HBM-budget admission.  Each result
is the same alone and in the mix; over-budget requests are rejected; a
request that cannot finish in time reports a timeout without losing it;
shutdown cancels what was not launched."""
import time

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import dev

pytestmark = pytest.mark.gpu


@pytest.fixture
def server(mmlib):
    """Re-initialises the library with given serving options, restores the
    defaults afterwards."""
    mm = mmlib

    def start(**kw):
        mm.mm_shutdown()
        st = mm.mm_init(device=0, **kw)
        assert st == mm.MM_OK
        return mm

    yield start
    mm.mm_shutdown()
    assert mm.mm_init(device=0) == mm.MM_OK


def _request_set(count, seed, lo=64, hi=700):
    t, dims, f64 = synth.serving_stream(seed, count, 1.0, lo, hi)
    reqs = []
    for k in range(count):
        n, m, p = (int(v) for v in dims[k])
        tdt = torch.float64 if f64[k] else torch.float32
        A = dev(synth.uniform_pm1(5000 + 2 * k, (n, m)), tdt)
        B = dev(synth.uniform_pm1(5001 + 2 * k, (m, p)), tdt)
        C = torch.full((n, p), float("nan"), dtype=tdt, device="cuda")
        reqs.append((n, m, p, A, B, C, bool(f64[k])))
    return reqs


def test_alone_equals_in_the_mix(server):
    mm = server(n_streams=3, max_batch=16, check=1)
    reqs = _request_set(60, 31)
    ids = []
    for (n, m, p, A, B, C, f64) in reqs:
        dt = mm.MM_F64 if f64 else mm.MM_F32
        st, rid = mm.mm_submit(n, m, p, A, B, C, dt, mm.MM_MODE_AUTO)
        assert st == mm.MM_OK
        ids.append(rid)
    lat = []
    for rid, (n, m, p, A, B, C, f64) in zip(ids, reqs):
        st, res, err, ms = mm.mm_wait(rid, 120.0)
        assert st == mm.MM_OK and res == mm.MM_OK
        tol = oracle.tolerance(m, "f64" if f64 else "f32")
        assert 0 <= err <= 4 * tol, (n, m, p, f64, err)
        lat.append(ms)
    st, done, batches, waiting, resident = mm.mm_serve_stats()
    # with nothing admitted, the bytes counted are the buffers the streams keep
    assert done == 60 and waiting == 0 and 0 <= resident <= 40 << 30 and batches >= 2
    # every result again, alone (a grouped call of that product only, the
    # path serving batches take): identical bits; and through mm_gemm, which
    # runs products with few tiles on the fused split-K kernel: within the
    # tolerance
    for (n, m, p, A, B, C, f64) in reqs:
        C1 = torch.full_like(C, float("nan"))
        dt = mm.MM_F64 if f64 else mm.MM_F32
        assert mm.mm_gemm_grouped([(n, m, p, A, B, C1)], dt, mm.MM_MODE_AUTO) == 0
        assert torch.equal(C, C1), (n, m, p, f64)
        C2 = torch.full_like(C, float("nan"))
        assert mm.mm_gemm(n, m, p, A, B, C2, dt, mm.MM_MODE_AUTO) == 0
        absref = (A.abs().double() @ B.abs().double()).cpu().numpy()
        e = oracle.rel_errors(C2.cpu().numpy(), C1.cpu().numpy(), absref).max()
        assert e <= oracle.tolerance(m, "f64" if f64 else "f32"), (n, m, p, f64, e)
    # and a sample of them against the oracle
    for k in range(0, 60, 6):
        n, m, p, A, B, C, f64 = reqs[k]
        ref, absref = oracle.default().gemm(A.cpu().numpy(), B.cpu().numpy(), with_abs=True)
        e = oracle.rel_errors(C.cpu().numpy(), ref, absref).max()
        assert e <= oracle.tolerance(m, "f64" if f64 else "f32")


def test_budget_admission(server):
    budget = 8 << 20
    mm = server(hbm_budget_bytes=budget, n_streams=2)
    big = 1100  # 3 * 1100^2 * 4 bytes > 8 MiB
    A = torch.zeros((big, big), device="cuda")
    st, _ = mm.mm_submit(big, big, big, A, A, A, mm.MM_F32, mm.MM_MODE_SPLIT_BF16X3)
    assert st == mm.MM_EBUDGET
    # many requests that each fit but not all together: all complete
    reqs = []
    for k in range(12):
        n = m = p = 400
        a = dev(synth.uniform_pm1(7000 + k, (n, m)))
        b = dev(synth.uniform_pm1(7100 + k, (m, p)))
        c = torch.zeros((n, p), device="cuda")
        st, rid = mm.mm_submit(n, m, p, a, b, c, mm.MM_F32, mm.MM_MODE_SPLIT_BF16X3)
        assert st == mm.MM_OK
        reqs.append((rid, a, b, c))
    for rid, a, b, c in reqs:
        st, res, _, _ = mm.mm_wait(rid, 120.0)
        assert st == mm.MM_OK and res == mm.MM_OK
    assert 0 <= mm.mm_serve_stats()[4] <= budget  # only the streams' kept buffers


def test_wait_timeout_then_result(server):
    mm = server(n_streams=1, max_batch=1)
    n = 4096
    A = torch.ones((n, n), dtype=torch.float64, device="cuda")
    C = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    st, rid = mm.mm_submit(n, n, n, A, A, C, mm.MM_F64, mm.MM_MODE_DGEMM)
    assert st == mm.MM_OK
    st, _, _, _ = mm.mm_wait(rid, 1e-4)  # far shorter than an FP64 4096^3 product
    assert st == mm.MM_ETIMEOUT
    st, res, _, _ = mm.mm_wait(rid, 120.0)
    assert st == mm.MM_OK and res == mm.MM_OK
    assert torch.all(C == float(n))
    assert mm.mm_poll(rid)[0] == mm.MM_ENOTFOUND  # reported once, then forgotten


def test_shutdown_cancels_unlaunched(server):
    mm = server(n_streams=1, max_batch=1)
    n = 2048
    A = torch.ones((n, n), dtype=torch.float64, device="cuda")
    outs, ids = [], []
    for k in range(8):
        C = torch.zeros((n, n), dtype=torch.float64, device="cuda")
        st, rid = mm.mm_submit(n, n, n, A, A, C, mm.MM_F64, mm.MM_MODE_DGEMM)
        assert st == mm.MM_OK
        outs.append(C)
        ids.append(rid)
        if k == 0:  # let the first request reach the GPU before the rest queue
            for _ in range(100000):
                if mm.mm_serve_stats()[2] >= 1:
                    break
            assert mm.mm_serve_stats()[2] >= 1
    assert mm.mm_shutdown() == mm.MM_OK
    results = [mm.mm_poll(r) for r in ids]
    assert all(r[0] == mm.MM_OK for r in results)
    codes = [r[1] for r in results]
    assert codes[0] == mm.MM_OK  # the first one was on the GPU already
    assert mm.MM_ECANCELLED in codes
    for c, code in zip(outs, codes):
        if code == mm.MM_OK:
            assert torch.all(c == float(n))


def test_submit_validation(server):
    mm = server()
    x = torch.zeros(4, device="cuda")
    h = np.zeros(4, np.float32)
    assert mm.mm_submit(2, 2, 2, h, x, x, mm.MM_F32, mm.MM_MODE_SIMT)[0] == mm.MM_EINVAL
    assert mm.mm_submit(-2, 2, 2, x, x, x, mm.MM_F32, mm.MM_MODE_SIMT)[0] == mm.MM_EINVAL
    assert mm.mm_submit(2, 2, 2, x, x, x, mm.MM_F64, mm.MM_MODE_SIMT)[0] == mm.MM_EUNSUPPORTED


def test_budget_counts_buffers_the_streams_keep(server):
    """A stream keeps the scratch of its largest batch for the next one.  Those
    bytes count against the budget, and an idle stream gives them back when
    the next request fits only without them: the reported total never exceeds
    the budget, and a request of nearly the whole budget still runs after a
    large split product left its buffers behind."""
    budget = 512 << 20
    mm = server(n_streams=1, hbm_budget_bytes=budget)
    n = 2048
    A = torch.rand(n, n, device="cuda") * 2 - 1
    B = torch.rand(n, n, device="cuda") * 2 - 1
    C = torch.empty(n, n, device="cuda")
    st, rid = mm.mm_submit(n, n, n, A, B, C, mm.MM_F32, mm.MM_MODE_SPLIT_BF16X3)
    assert st == mm.MM_OK
    st, res, _, _ = mm.mm_wait(rid, 60.0)
    assert st == mm.MM_OK and res == mm.MM_OK
    _, _, _, _, held = mm.mm_serve_stats()
    assert 0 < held <= budget, held  # the split packs of 2048^3, kept by the stream
    # SIMT requests carry no scratch estimate: operands and output alone, here
    # budget - 16 MiB, which fits only once the stream's buffers are gone
    x = int(((budget - (16 << 20)) / 12) ** 0.5)
    assert 12 * x * x + held > budget
    A2 = torch.rand(x, x, device="cuda") * 2 - 1
    B2 = torch.rand(x, x, device="cuda") * 2 - 1
    C2 = torch.empty(x, x, device="cuda")
    st, rid = mm.mm_submit(x, x, x, A2, B2, C2, mm.MM_F32, mm.MM_MODE_SIMT)
    assert st == mm.MM_OK
    peak = 0
    for _ in range(2000):
        st, res, _, _ = mm.mm_poll(rid)
        _, _, _, _, r = mm.mm_serve_stats()
        peak = max(peak, r)
        if st == mm.MM_OK:
            break
        time.sleep(0.005)
    else:
        st, res, _, _ = mm.mm_wait(rid, 120.0)
    assert st == mm.MM_OK and res == mm.MM_OK
    assert peak <= budget, peak
    I, J = synth.sample_indices(77, x, x, 64)
    hi, lo, ab = oracle.default().entries(A2.cpu().numpy(), B2.cpu().numpy(), I, J)
    got = C2.cpu().numpy()[I, J].astype(np.float64)
    assert oracle.rel_errors(got, hi + lo, ab).max() <= oracle.tolerance(x, "f32")
