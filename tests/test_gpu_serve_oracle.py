"""The serving workload at its stated scale against the CPU FP64 oracle:
50,000 requests with dims log-uniform in [64, 4096] (rounded), 20% FP64 on
the Ozaki path with its accuracy gate and 80% FP32 on the split-BF16x3 path,
operands resident on the device, admission under the default 40 GiB budget,
submitted as fast as the library admits them.  A 1% sample of the requests
(every 100th, 500 in all) keeps 1024 seeded output entries each, and each of
those is compared with the oracle's compensated (Dot2) value under the
elementwise metric e_ij = |c^_ij - c_ij| / (|A||B|)_ij: at most 1e-6 sqrt(m)
for FP32 requests and 1e-14 sqrt(m) for FP64 requests; sampled requests whose
C has at most 2^20 entries also keep all of C for a Freivalds check by the
oracle ((A B) x against A (B x), normalised by |A| (|B| |x|), within 4 times
the tolerance).  The operands of request k are prefixes of two seeded device
buffers, as in the serving benchmark, so the host holds one copy of each for
the oracle."""
import collections
import time

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

COUNT = 50000
EVERY = 100       # the 1% sample
ENTRIES = 1024    # sampled output entries per sampled request
FULL_MAX = 1 << 20  # sampled requests with at most this many outputs keep all of C
OUT_CAP = 16 << 30  # outstanding output bytes the client holds at most


@pytest.fixture
def serving(mmlib):
    mm = mmlib
    mm.mm_shutdown()
    assert mm.mm_init(device=0, n_streams=2) == mm.MM_OK
    yield mm
    mm.mm_shutdown()
    assert mm.mm_init(device=0) == mm.MM_OK


def test_serving_workload_against_oracle(serving):
    mm = serving
    _, dims, f64 = synth.serving_stream(5, COUNT, 1.0)
    big = 4096 * 4096
    h32 = synth.uniform_pm1(91, (big,)).astype(np.float32)
    h64 = synth.uniform_pm1_f64(92, (big,))
    src32 = torch.from_numpy(h32).cuda()
    src64 = torch.from_numpy(h64).cuda()

    live = collections.OrderedDict()  # request id -> (k, C)
    kept = {}  # k -> (I, J, sampled entries of C, all of C or None)
    held = [0]

    def finish(rid):
        k, C = live.pop(rid)
        held[0] -= C.numel() * C.element_size()
        if k % EVERY == 0:
            n, _, p = (int(v) for v in dims[k])
            I, J = synth.sample_indices(1000 + k, n, p, ENTRIES)
            Ct = C.view(n, p)
            kept[k] = (I, J, Ct[torch.from_numpy(I).cuda(), torch.from_numpy(J).cuda()]
                       .double().cpu().numpy(),
                       Ct.double().cpu().numpy() if n * p <= FULL_MAX else None)

    def drain(budget=64):
        done = []
        for rid in list(live)[:budget]:
            st, res, _, _ = mm.mm_poll(rid)
            if st == mm.MM_OK:
                assert res == mm.MM_OK, mm.mm_strerror(res)
                done.append(rid)
        for rid in done:
            finish(rid)

    t0 = time.perf_counter()
    for k in range(COUNT):
        n, m, p = (int(v) for v in dims[k])
        if f64[k]:
            A, B, dt, md = src64[:n * m], src64[:m * p], mm.MM_F64, mm.MM_MODE_OZAKI
            C = torch.empty(n * p, device="cuda", dtype=torch.float64)
        else:
            A, B, dt, md = src32[:n * m], src32[:m * p], mm.MM_F32, mm.MM_MODE_SPLIT_BF16X3
            C = torch.empty(n * p, device="cuda")
        while live and held[0] + C.numel() * C.element_size() > OUT_CAP:
            drain()
        st, rid = mm.mm_submit(n, m, p, A, B, C, dt, md)
        assert st == mm.MM_OK, mm.mm_strerror(st)
        live[rid] = (k, C)
        held[0] += C.numel() * C.element_size()
    while live:
        drain()
    wall = time.perf_counter() - t0
    assert len(kept) == COUNT // EVERY

    orc = oracle.default()
    worst = {False: 0.0, True: 0.0}  # max e_ij / tolerance per class
    emax = {False: 0.0, True: 0.0}
    fre = {False: 0.0, True: 0.0}  # max Freivalds ratio / tolerance per class
    for k, (I, J, got, full) in kept.items():
        n, m, p = (int(v) for v in dims[k])
        src = h64 if f64[k] else h32
        A = src[:n * m].reshape(n, m)
        B = src[:m * p].reshape(m, p)
        hi, lo, ab = orc.entries(A, B, I, J, "dot2")
        e = oracle.rel_errors(got, hi + lo, ab)
        tol = oracle.tolerance(m, "f64" if f64[k] else "f32")
        emax[bool(f64[k])] = max(emax[bool(f64[k])], float(e.max()))
        worst[bool(f64[k])] = max(worst[bool(f64[k])], float(e.max()) / tol)
        if full is not None:
            x = synth.freivalds_vector(2000 + k, p)
            y, _ = orc.gemv(full, x)
            z, za = orc.freivalds_rhs(A, B, x)
            r = np.abs(y - z) / np.where(za > 0, za, 1.0)
            fre[bool(f64[k])] = max(fre[bool(f64[k])], float(r.max()) / tol)
    print("\nserving %d requests in %.1f s (%.0f req/s); 1%% sample: FP32 max e %.3g "
          "(%.3g of tol), FP64 max e %.3g (%.3g of tol); Freivalds / tol FP32 %.3g, FP64 %.3g"
          % (COUNT, wall, COUNT / wall, emax[False], worst[False], emax[True], worst[True],
             fre[False], fre[True]))
    assert worst[False] <= 1.0 and worst[True] <= 1.0
    assert fre[False] <= 4.0 and fre[True] <= 4.0
