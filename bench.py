"""Benchmark of the dense product C = A.B on GB300.

One step = one split-BF16x3 product (operand scaling + hi/lo packing +
tcgen05 tensor-core GEMM) of the square FP32 workload n = m = p = 8192,
entries uniform[-1,1) from seeds 0 (A) and 1 (B), through the C ABI on
device-resident operands (inputs larger than L2: 268 MB per operand and per
packed operand).  Metric: useful TFLOP/s = 2 n m p / time.

Also reported on the same line: the plain SIMT FP32 and FP64 paths at the
same size (the split path's target is >= 3x the SIMT rate), the dominant
kernel's roofline, the end-to-end rate through mm_gemm with pinned host
buffers, the CPU oracle's rate on a bounded sample, clocks during the timed
region, and the count of library kernel launches.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mine|reference]

--impl reference times the CPU oracle (the FP64 evaluation of the definition
in Listing 1's order) on a bounded sample of the same workload: there is no
reference implementation of this GPU path to run.
Multi-GPU (torchrun): every rank runs its own product (independent problems,
weak scaling); no collective touches the data, only a barrier and a max of
the times.  With --shard rows one product is split by row blocks of A and C
over the ranks instead (strong scaling; B replicated; the gather of C is
timed apart from the product).
"""
from __future__ import annotations

import argparse
import collections
import itertools
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_DEFAULT = 8192


def workload(n: int) -> str:
    return "square FP32 GEMM n=m=p=%d, uniform[-1,1) seeds 0/1" % n


def workload_config(n: int, world: int) -> dict:
    """The workload both arms run (the same dict in the reference arm's line);
    the method that computes it is the line's "path"."""
    mb = 4 * n * n / 1e6
    l2 = ("inputs larger than L2 (%.0f MB per operand)" % mb if mb > 129
          else "operands of %.1f MB each (within L2)" % mb)
    return {"workload": workload(n), "n": n, "m": n, "p": n, "l2": l2,
            "parallelism": "replicas x%d" % world}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def whole_job_rate(units_per_rank: float, world: int, max_ms: float) -> float:
    """Whole-job throughput: the units all ranks processed / the slowest
    rank's time (weak scaling: every rank does the same work)."""
    return world * units_per_rank / (max_ms * 1e-3)


def max_over_ranks(ms: float, dist, device=None) -> float:
    """Max of a per-rank time over the process group (identity without one)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.path or not os.path.exists(self.path):
            return out
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[4:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return out
        loaded = [r for r in rows if r[2] > 300.0] or rows
        out["sm_mhz"] = statistics.median(r[0] for r in loaded)
        out["sm_max_mhz"] = max(r[1] for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        seen = set()
        for r in loaded:
            for name, v in zip(names, r[3][1:]):
                if v.lower().startswith("active"):
                    seen.add(name)
        out["reasons"] = sorted(seen)
        out["samples"] = len(loaded)
        out["power_w_max"] = max(r[2] for r in rows)
        return out


class OracleSampler:
    """The FP64 CPU oracle (all host cores, Listing 1 order) on a block of
    rows of the n x n x n workload: the same B, the first `rows` rows of A."""

    def __init__(self, n: int):
        import numpy as np

        import oracle
        import synth
        self.n = n
        self.orc = oracle.default()
        self.cores = self.orc.default_threads()
        self.B = synth.uniform_pm1(1, (n, n)).astype(np.float64)
        self.A = None

    def run(self, rows: int) -> float:
        import numpy as np

        import synth
        if self.A is None or self.A.shape[0] != rows:
            self.A = synth.uniform_pm1(0, (rows, self.n)).astype(np.float64)
        t0 = time.perf_counter()
        self.orc.gemm(self.A, self.B, threads=self.cores)
        return time.perf_counter() - t0

    def calibrate(self, target_s: float, cap_rows: int = 4096) -> int:
        """Row count whose run takes about target_s seconds."""
        cap_rows = min(cap_rows, self.n)
        rows = min(max(self.cores, 8), cap_rows)
        t = self.run(rows)
        while t < 0.25 * target_s and rows < cap_rows:
            rows = min(cap_rows, rows * 4)
            t = self.run(rows)
        return int(min(cap_rows, max(min(8, cap_rows), rows * target_s / max(t, 1e-3))))

    def flops(self, rows: int) -> float:
        return 2.0 * rows * self.n * self.n


def oracle_sample_rate(n: int, target_s: float = 12.0):
    """(TFLOP/s, cores, rows, seconds) of one oracle sample of ~target_s."""
    smp = OracleSampler(n)
    rows = smp.calibrate(target_s)
    t = smp.run(rows)
    return smp.flops(rows) / t / 1e12, smp.cores, rows, t


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    n = args.size
    smp = OracleSampler(n)
    # every step is a bounded sample: the whole run stays within a few minutes
    per_step = min(6.0, max(0.3, 150.0 / max(args.steps, 1)))
    rows = smp.calibrate(per_step)
    for _ in range(args.warmup):
        smp.run(rows)
    times = [smp.run(rows) for _ in range(args.steps)]
    value = smp.flops(rows) * len(times) / sum(times) / 1e12
    sample = "%d of %d rows of C per step (FP64 oracle, Listing 1 order, %d threads)" % (
        rows, n, smp.cores)
    line = {
        "impl": "reference", "metric": "GEMM TFLOP/s", "value": value, "unit": "TFLOP/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "path": "CPU FP64 oracle",
        "config": workload_config(n, world),
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": smp.cores,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def _traffic_from_profiles(name: str):
    """DRAM bytes per launch of a kernel from its committed ncu summary
    (a line 'dram_bytes_per_launch: <int>' with the command that made it)."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        for line in open(path):
            if line.startswith("dram_bytes_per_launch:"):
                return float(line.split(":", 1)[1].split()[0])
    except (OSError, ValueError):
        pass
    return None


def gpu_check(mm, n, m, p, A, B, C, dt, seed=2, samples=4096):
    """The library's FP64 GPU check of a computed product: (Freivalds max
    normalised residual, max normalised error on sampled entries)."""
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    x = torch.rand(p, device="cuda", dtype=torch.float64, generator=g) * 2 - 1
    I = torch.randint(0, n, (samples,), device="cuda", generator=g)
    J = torch.randint(0, p, (samples,), device="cuda", generator=g)
    st, fr, sm = mm.mm_check(n, m, p, A, B, C, dt, x, I, J)
    mm.check_status(st, "mm_check")
    return fr, sm


def bench_paper_workloads(mm, stream, peaks, n: int = 4096, reps: int = 5):
    """The paper's Table 2 products at its size (4096 x 4096: float, double,
    complex float), in seconds per product beside the paper's fastest device
    (Tesla C2050 with shared memory: 0.83 s, 1.6 s, 2.07 s), and its matrix
    addition plus the diagonal special case as HBM bandwidth."""
    import torch
    gen = torch.Generator(device="cuda")
    gen.manual_seed(0)
    A = torch.rand((n, n), device="cuda", generator=gen) * 2 - 1
    B = torch.rand((n, n), device="cuda", generator=gen) * 2 - 1
    C = torch.empty((n, n), device="cuda")

    def t_ms(fn):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps * 1e3

    ok = lambda st, w: mm.check_status(st, w)
    out = {"n": n}
    out["float_split_s"] = t_ms(lambda: ok(mm.mm_gemm(n, n, n, A, B, C, mm.MM_F32,
                                                      mm.MM_MODE_SPLIT_BF16X3), "f")) / 1e3
    out["float_simt_s"] = t_ms(lambda: ok(mm.mm_gemm(n, n, n, A, B, C, mm.MM_F32,
                                                     mm.MM_MODE_SIMT), "s")) / 1e3
    A64, B64 = A.double(), B.double()
    C64 = torch.empty((n, n), device="cuda", dtype=torch.float64)
    out["double_s"] = t_ms(lambda: ok(mm.mm_gemm(n, n, n, A64, B64, C64, mm.MM_F64,
                                                 mm.MM_MODE_DGEMM), "d")) / 1e3
    del A64, B64, C64
    Az = torch.complex(A, B)
    Bz = torch.complex(B, A)
    Cz = torch.empty((n, n), device="cuda", dtype=torch.complex64)
    out["complex_float_s"] = t_ms(lambda: ok(mm.mm_cgemm(n, n, n, Az, Bz, Cz,
                                                         mm.MM_MODE_SPLIT_BF16X3), "c")) / 1e3
    out["complex_float_tflops"] = 8.0 * n ** 3 / out["complex_float_s"] / 1e12
    del Az, Bz, Cz
    out["paper_c2050_shared_s"] = {"float": 0.83, "double": 1.6, "complex_float": 2.07}
    hbm = peaks.get("hbm_gbs", 6800.0)
    d = A[0].contiguous()

    def kernel_ms(name, fn):
        # device time of the library's kernel (tracer events on its stream)
        fn()
        mm.mm_trace_reset()
        mm.mm_trace_enable(True)
        for _ in range(reps):
            fn()
        mm.mm_trace_enable(False)
        _, k, tot = mm.mm_trace_read(name)
        mm.mm_trace_reset()
        return tot / max(k, 1)

    def queued_ms(fn, k=20):
        # asynchronous calls queued back to back on one stream, timed by events
        # around all of them: kernel time without a synchronous call's launch
        # latency
        fn()
        mm.check_status(mm.mm_sync(stream), "sync")
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    ms = kernel_ms("add", lambda: ok(mm.mm_add(n, n, 1.0, A, -1.0, B, C, mm.MM_F32), "add"))
    out["add_gbs"] = 3 * 4 * n * n / (ms * 1e-3) / 1e9
    out["add_frac_hbm"] = out["add_gbs"] / hbm
    ms = kernel_ms("diag", lambda: ok(mm.mm_diag(n, n, A, d, C, 0, mm.MM_F32), "diag"))
    out["diag_gbs"] = (2 * 4 * n * n + 4 * n) / (ms * 1e-3) / 1e9
    out["diag_frac_hbm"] = out["diag_gbs"] / hbm
    ms = queued_ms(lambda: ok(mm.mm_add_async(n, n, 1.0, A, -1.0, B, C, mm.MM_F32, stream), "add"))
    out["add_gbs_queued"] = 3 * 4 * n * n / (ms * 1e-3) / 1e9
    out["add_frac_hbm_queued"] = out["add_gbs_queued"] / hbm
    ms = queued_ms(lambda: ok(mm.mm_diag_async(n, n, A, d, C, 0, mm.MM_F32, stream), "diag"))
    out["diag_gbs_queued"] = (2 * 4 * n * n + 4 * n) / (ms * 1e-3) / 1e9
    out["diag_frac_hbm_queued"] = out["diag_gbs_queued"] / hbm
    # the product with the matrix subtraction C = A.B - D: as two calls (the
    # product, then mm_add over C and D) and with the subtraction fused into
    # the product's epilogue (mm_gemm_axpby: D read once as C is stored)
    F32, X3 = mm.MM_F32, mm.MM_MODE_SPLIT_BF16X3

    def two_calls():
        ok(mm.mm_gemm_async(n, n, n, A, B, C, F32, X3, stream), "gemm")
        ok(mm.mm_add_async(n, n, 1.0, C, -1.0, B, C, F32, stream), "add")

    out["gemm_then_add_ms"] = queued_ms(two_calls)
    out["gemm_axpby_fused_ms"] = queued_ms(
        lambda: ok(mm.mm_gemm_axpby_async(n, n, n, 1.0, A, B, -1.0, B, C, F32, X3, stream), "axpby"))
    out["gemm_only_ms"] = queued_ms(lambda: ok(mm.mm_gemm_async(n, n, n, A, B, C, F32, X3, stream),
                                               "gemm"))
    # the same kernels on 8192^2 operands, where the ~10 us between a synchronous
    # call's first trace event and its kernel weighs less
    del A, B, C
    n2 = 2 * n
    A2 = torch.rand((n2, n2), device="cuda", generator=gen)
    B2 = torch.rand((n2, n2), device="cuda", generator=gen)
    C2 = torch.empty((n2, n2), device="cuda")
    d2 = A2[0].contiguous()
    ms = kernel_ms("add", lambda: ok(mm.mm_add(n2, n2, 1.0, A2, -1.0, B2, C2, mm.MM_F32), "add"))
    out["add_gbs_%d" % n2] = 3 * 4 * n2 * n2 / (ms * 1e-3) / 1e9
    out["add_frac_hbm_%d" % n2] = out["add_gbs_%d" % n2] / hbm
    ms = kernel_ms("diag", lambda: ok(mm.mm_diag(n2, n2, A2, d2, C2, 0, mm.MM_F32), "diag"))
    out["diag_gbs_%d" % n2] = (2 * 4 * n2 * n2 + 4 * n2) / (ms * 1e-3) / 1e9
    out["diag_frac_hbm_%d" % n2] = out["diag_gbs_%d" % n2] / hbm
    del A2, B2, C2
    out["note"] = ("products: synchronous calls timed on the host; add / diag: time from the "
                   "library's event tracer, which includes the launch latency of a synchronous "
                   "call (~10 us); *_queued: 20 asynchronous calls queued on one stream, timed "
                   "by events around all of them; add moves 192 MB (768 MB at 8192^2) and diag "
                   "128 MB (512 MB) per call; gemm_then_add / gemm_axpby_fused / gemm_only: "
                   "C = A.B - D at 4096^3 on the split path, queued, per call")
    return out


def bench_stress(mm, stream, peaks, reps: int = 10):
    """Config 3, shape and value stress with FP32 in/out: the rectangular
    8192x512.512x8192 product (TFLOP/s), the skinny 64x16384.16384x64 one
    (bandwidth-bound: GB/s of A + B + C against the measured HBM copy rate,
    64 operand copies taken round-robin so the 512 MB footprint exceeds L2),
    B = diag(d) at 4096 through the general product, and 4096^3 with entries
    s 2^e, e real uniform in [-20, 20) (split-precision scaling; FP8 error
    reported).  Device time per product from CUDA events on the stream, the
    calls queued behind a device-side wait so that their submission does not
    gate them; the library's FP64 check for the error.  A failure is
    recorded, not raised."""
    import torch

    import synth
    out = {}
    hbm = peaks.get("hbm_gbs", 6797.9)

    def per_call_ms(fn, count, warm=2):
        for k in range(warm):
            fn(k)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        # the calls are queued behind a ~10 ms device-side wait, so that the
        # host's submission of short products does not gate the device time
        with torch.cuda.stream(stream):
            torch.cuda._sleep(20_000_000)
        e0.record(stream)
        for k in range(count):
            fn(k)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / count

    def gemm(n, m, p, A, B, C, md):
        mm.check_status(mm.mm_gemm_async(n, m, p, A, B, C, mm.MM_F32, md, stream), "stress")

    modes = (("simt", mm.MM_MODE_SIMT), ("split", mm.MM_MODE_SPLIT_BF16X3))
    try:
        gen = torch.Generator(device="cuda")
        gen.manual_seed(3)
        # 3a: rectangular, a large C write
        n, m, p = 8192, 512, 8192
        A = torch.rand(n, m, device="cuda", generator=gen) * 2 - 1
        B = torch.rand(m, p, device="cuda", generator=gen) * 2 - 1
        C = torch.empty(n, p, device="cuda")
        for name, md in modes:
            ms = per_call_ms(lambda k: gemm(n, m, p, A, B, C, md), reps)
            out["rect_8192x512x8192_" + name] = {
                "ms": ms, "tflops": 2.0 * n * m * p / (ms * 1e-3) / 1e12,
                "gbs": 4.0 * (n * m + m * p + n * p) / (ms * 1e-3) / 1e9}
        out["rect_check_split"] = gpu_check(mm, n, m, p, A, B, C, mm.MM_F32)
        del A, B, C
        # 3b: skinny, bandwidth-bound
        n, m, p, copies = 64, 16384, 64, 64
        As = torch.rand(copies, n, m, device="cuda", generator=gen) * 2 - 1
        Bs = torch.rand(copies, m, p, device="cuda", generator=gen) * 2 - 1
        Cs = torch.empty(copies, n, p, device="cuda")
        nbytes = 4.0 * (n * m + m * p + n * p)
        for name, md in modes:
            ms = per_call_ms(lambda k: gemm(n, m, p, As[k % copies], Bs[k % copies],
                                            Cs[k % copies], md), 4 * copies)
            gbs = nbytes / (ms * 1e-3) / 1e9
            out["skinny_64x16384x64_" + name] = {"us": ms * 1e3, "gbs": gbs, "frac_hbm": gbs / hbm}
        out["skinny_check_split"] = gpu_check(mm, n, m, p, As[0], Bs[0], Cs[0], mm.MM_F32)
        _, tiles, sl, ql, csz = mm.mm_tune_query_splitk(n, m, p)
        out["skinny_split_path"] = ("fused split-K: %d slices in %d clusters of %d" % (sl, ql, csz)
                                    if sl else "packed")
        del As, Bs, Cs
        # 3c: B = diag(d) through the general product (dense flops counted)
        n = 4096
        A = torch.rand(n, n, device="cuda", generator=gen) * 2 - 1
        Bd = torch.diag(torch.rand(n, device="cuda", generator=gen) * 2 - 1).contiguous()
        C = torch.empty(n, n, device="cuda")
        for name, md in modes:
            ms = per_call_ms(lambda k: gemm(n, n, n, A, Bd, C, md), reps)
            out["diag_4096_" + name] = {"ms": ms, "dense_tflops": 2.0 * n ** 3 / (ms * 1e-3) / 1e12}
        del A, Bd, C
        # 3d/3e: s 2^e entries, e real in [-20, 20)
        A = torch.from_numpy(synth.pow2_real(30, (n, n))).cuda()
        B = torch.from_numpy(synth.pow2_real(31, (n, n))).cuda()
        C = torch.empty(n, n, device="cuda")
        ms = per_call_ms(lambda k: gemm(n, n, n, A, B, C, mm.MM_MODE_SPLIT_BF16X3), reps)
        out["pow2_4096_split"] = {"ms": ms, "tflops": 2.0 * n ** 3 / (ms * 1e-3) / 1e12,
                                  "check": gpu_check(mm, n, n, n, A, B, C, mm.MM_F32)}
        gemm(n, n, n, A, B, C, mm.MM_MODE_FP8)
        mm.check_status(mm.mm_sync(stream), "stress fp8")
        out["pow2_4096_fp8_check"] = gpu_check(mm, n, n, n, A, B, C, mm.MM_F32)
        del A, B, C
    except Exception as ex:  # recorded in the JSON line instead of ending the run
        out["error"] = repr(ex)
    return out


def bench_grouped(mm, stream, steps: int, seed: int = 4, count: int = 4096):
    """Grouped GEMM of `count` products, n, m, p uniform over {32, ..., 1024}
    step 32 (seeded), split path: one grouped launch per step vs one launch
    per product.  Returns a dict of TFLOP/s and launch counts."""
    import torch

    import synth
    dims = synth.grouped_dims(seed, count)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    probs = []
    flops = 0.0
    for (n, m, p) in dims:
        n, m, p = int(n), int(m), int(p)
        A = torch.rand((n, m), device="cuda", generator=gen) * 2 - 1
        B = torch.rand((m, p), device="cuda", generator=gen) * 2 - 1
        C = torch.empty((n, p), device="cuda")
        probs.append((n, m, p, A, B, C))
        flops += 2.0 * n * m * p
    md = mm.MM_MODE_SPLIT_BF16X3

    table = mm.mm_problems(probs)  # marshalled once, outside the timing

    def grouped():
        mm.check_status(mm.mm_gemm_grouped_async(table, mm.MM_F32, md, stream), "grouped")

    def singles():
        for (n, m, p, A, B, C) in probs:
            mm.check_status(mm.mm_gemm_async(n, m, p, A, B, C, mm.MM_F32, md, stream), "single")

    out = {"instances": count, "tflop": flops / 1e12}
    for name, fn, k in (("grouped", grouped, steps), ("per_instance", singles, max(1, steps // 4))):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        l0 = mm.mm_launch_count()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / k
        out[name + "_tflops"] = flops / (ms * 1e-3) / 1e12
        out[name + "_ms"] = ms
        out[name + "_launches_per_step"] = (mm.mm_launch_count() - l0) / k
    mm.check_status(mm.mm_sync(stream), "grouped sync")
    # device time of each kernel of one grouped step (the library's tracer)
    mm.mm_trace_reset()
    mm.mm_trace_enable(True)
    grouped()
    mm.check_status(mm.mm_sync(stream), "grouped traced run")
    mm.mm_trace_enable(False)
    out["grouped_kernels_ms"] = {}
    for kname in ("split_maps", "split_pack", "split_verify", "split_fix", "split_tc"):
        _, cnt, kms = mm.mm_trace_read(kname)
        if cnt:
            out["grouped_kernels_ms"][kname] = kms
    mm.mm_trace_reset()
    # every instance: the library's FP64 GPU check, one Freivalds vector and 64
    # sampled entries, each against its own tolerance 1e-6 sqrt(m)
    grouped()
    mm.check_status(mm.mm_sync(stream), "grouped check run")
    worst, worst_ratio, over = 0.0, 0.0, 0
    for g, (n, m, p, A, B, C) in enumerate(probs):
        fr, sm = gpu_check(mm, n, m, p, A, B, C, mm.MM_F32, seed=100 + g, samples=64)
        e = max(fr, sm)
        tol = 1e-6 * m ** 0.5
        worst = max(worst, e)
        worst_ratio = max(worst_ratio, e / tol)
        over += int(e > tol)
    out["check_all"] = {"instances": len(probs), "max_err": worst,
                        "max_err_over_tol": worst_ratio, "over_tol": over,
                        "check": "per instance: 1 Freivalds vector + 64 sampled entries (FP64, GPU)"}
    del probs
    return out


def bench_serving(mm, count: int, rate_frac: float, seed: int = 5, streams: int = 2,
                  max_batch: int = 0, capacity=None, f64_mode=None, check: bool = False):
    """Poisson replay of `count` requests (dims log-uniform in [64, 4096], 20%
    FP64) through mm_submit/mm_poll with operands resident on the device.
    f64_mode: the path of the FP64 requests (default MM_MODE_DGEMM).
    The arrival rate is rate_frac x the measured capacity (requests/s of the
    same mix submitted all at once).  Returns p50/p99 latency (all requests and
    per class: FP32 on the split path, FP64) and rates; with check=True the
    serving loop also runs the library's FP64 GPU check (Freivalds + 64
    sampled entries) on every result and the maximum normalised error of each
    class is returned beside its tolerance's worst case over the mix."""
    import numpy as np
    import torch

    import synth
    _, dims, f64 = synth.serving_stream(seed, count, 1.0)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    big = 4096 * 4096
    src32 = torch.rand(big, device="cuda", generator=gen) * 2 - 1
    src64 = src32.double()

    f64_md = mm.MM_MODE_DGEMM if f64_mode is None else f64_mode
    out_cap = 40 << 30  # the client's outstanding output bytes (backpressure)
    held = [0]

    def submit(k):
        n, m, p = (int(v) for v in dims[k])
        if f64[k]:
            A, B, dt, md = src64[:n * m], src64[:m * p], mm.MM_F64, f64_md
            C = torch.empty(n * p, device="cuda", dtype=torch.float64)
        else:
            A, B, dt, md = src32[:n * m], src32[:m * p], mm.MM_F32, mm.MM_MODE_SPLIT_BF16X3
            C = torch.empty(n * p, device="cuda")
        st, rid = mm.mm_submit(n, m, p, A, B, C, dt, md)
        mm.check_status(st, "mm_submit")
        held[0] += C.numel() * C.element_size()
        cls[rid] = (bool(f64[k]), m)
        return rid, C

    cls = {}          # request id -> (is FP64, inner dimension)
    err_max = {False: 0.0, True: 0.0}
    err_ratio = {False: 0.0, True: 0.0}  # error / tolerance of the request

    def drain(live, lat, budget=32):
        # polls the oldest requests first, a bounded number per call
        done = []
        for rid in itertools.islice(live, budget):
            st, res, err, ms = mm.mm_poll(rid)
            if st == mm.MM_OK:
                mm.check_status(res, "request")
                is64, mk = cls.pop(rid)
                lat.append((ms, is64))
                if check:
                    tol = (1e-14 if is64 else 1e-6) * max(mk, 1) ** 0.5
                    err_max[is64] = max(err_max[is64], err)
                    err_ratio[is64] = max(err_ratio[is64], err / tol)
                done.append(rid)
        for rid in done:
            C = live.pop(rid)
            held[0] -= C.numel() * C.element_size()

    def make_room(live, lat, k):
        n, _, p = (int(v) for v in dims[k])
        need = n * p * (8 if f64[k] else 4)
        while live and held[0] + need > out_cap:
            drain(live, lat)

    flops = float(np.sum(2.0 * dims[:, 0] * dims[:, 1] * dims[:, 2]))
    dev_index = torch.cuda.current_device()
    mm.mm_shutdown()
    mm.check_status(mm.mm_init(n_streams=streams, max_batch=max_batch, device=dev_index,
                               check=1 if check else 0), "mm_init serving")
    if capacity is None:
        # capacity: everything submitted at once
        live, lat = collections.OrderedDict(), []
        t0 = time.perf_counter()
        for k in range(count):
            make_room(live, lat, k)
            rid, C = submit(k)
            live[rid] = C
        while live:
            drain(live, lat)
        capacity = count / (time.perf_counter() - t0)
    rate = rate_frac * capacity
    gaps = -np.log1p(-synth.uniform01_f64(seed + 1, count)) / rate
    arrivals = np.cumsum(gaps)
    live, lat = collections.OrderedDict(), []
    t0 = time.perf_counter()
    for k in range(count):
        while time.perf_counter() - t0 < arrivals[k]:
            drain(live, lat)
        make_room(live, lat, k)
        rid, C = submit(k)
        live[rid] = C
    while live:
        drain(live, lat)
    wall = time.perf_counter() - t0
    st, completed, batches, waiting, resident = mm.mm_serve_stats()
    mm.mm_shutdown()
    mm.check_status(mm.mm_init(device=dev_index), "mm_init default")
    ms_all = np.asarray([x[0] for x in lat])
    out = {"requests": count, "rate_req_s": rate, "capacity_req_s": capacity,
           "p50_ms": float(np.percentile(ms_all, 50)), "p99_ms": float(np.percentile(ms_all, 99)),
           "throughput_req_s": count / wall, "tflops": flops / wall / 1e12,
           "batches": batches, "streams": streams, "max_batch": max_batch or 256}
    for name, want in (("f32_split", False), ("f64", True)):
        v = np.asarray([x[0] for x in lat if x[1] == want])
        if v.size:
            out[name] = {"requests": int(v.size), "p50_ms": float(np.percentile(v, 50)),
                         "p99_ms": float(np.percentile(v, 99))}
            if check:
                out[name]["max_err"] = err_max[want]
                out[name]["max_err_over_tol"] = err_ratio[want]
    return out


def run_grouped_only(args):
    """Only the grouped leg (config 4) with --grouped-count instances (the
    first ones of the seeded 4096-instance workload): grouped launch vs one
    launch per instance.  Prints one JSON line; also the profiling driver of
    the grouped tensor-core kernel."""
    import torch

    import paper_1306_6192_gb300 as mm
    torch.cuda.set_device(0)
    mm.check_status(mm.mm_init(device=0), "mm_init")
    stream = torch.cuda.Stream()
    out = bench_grouped(mm, stream, max(1, args.steps), count=args.grouped_count)
    mm.mm_shutdown()
    print(json.dumps({"metric": "grouped GEMM TFLOP/s", "grouped": out}))
    return 0


# the emulation's kernels as the library's tracer names them: maxima, digit
# slices, level products, exact sum; then the accuracy gate (its own kernels,
# its split-path product, and the FP64 FMA kernel that returns at once unless
# the gate failed)
OZAKI_TRACE = ("ozaki_max", "ozaki_digits", "split_maps", "fp8_tc", "ozaki_sum", "ozaki_gate",
               "split_pack", "split_verify", "split_fix", "split_tc", "dgemm_f64")


def run_fp8_only(args):
    """Only the FP8 e4m3 product (per-block scales) at n = m = p = --size on
    uniform[-1,1) operands (seeds 0/1): step rate, per-kernel device time and
    the library's FP64 check of the result.  Prints one JSON line; also the
    profiling driver of the FP8 kernels."""
    import torch

    import paper_1306_6192_gb300 as mm
    import synth
    torch.cuda.set_device(0)
    mm.check_status(mm.mm_init(device=0), "mm_init")
    n = args.size
    A = torch.from_numpy(synth.uniform_pm1(0, (n, n))).cuda()
    B = torch.from_numpy(synth.uniform_pm1(1, (n, n))).cuda()
    C = torch.empty((n, n), device="cuda")
    stream = torch.cuda.Stream()
    run = lambda: mm.check_status(mm.mm_gemm_async(n, n, n, A, B, C, mm.MM_F32, mm.MM_MODE_FP8,
                                                   stream), "fp8")
    for _ in range(args.warmup):
        run()
    torch.cuda.synchronize()
    mm.mm_trace_reset()
    mm.mm_trace_enable(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        run()
    e1.record(stream)
    torch.cuda.synchronize()
    mm.mm_trace_enable(False)
    ms = e0.elapsed_time(e1) / args.steps
    kernels = {}
    for k in ("fp8_max", "fp8_pack", "fp8_tc", "fp8_blk"):
        _, cnt, kms = mm.mm_trace_read(k)
        if cnt:
            kernels[k] = kms / cnt
    check = gpu_check(mm, n, n, n, A, B, C, mm.MM_F32)
    mm.mm_shutdown()
    flops = 2.0 * n ** 3
    out = {"metric": "FP8 e4m3 GEMM TFLOP/s (per-block scales)", "value": flops / (ms * 1e-3) / 1e12,
           "unit": "TFLOP/s", "n": n, "ms": ms, "steps": args.steps, "kernels_ms": kernels,
           "check": check}
    # the tensor-core kernel that computed the product: the 128 x 256 one when
    # every tile keeps one exponent along K, else the blockwise one (the other
    # returns at once)
    k_ms = kernels.get("fp8_tc", 0.0) + kernels.get("fp8_blk", 0.0)
    if k_ms > 0:
        out["tc_tflops"] = flops / (k_ms * 1e-3) / 1e12
    print(json.dumps(out))
    return 0


def run_ozaki_only(args):
    """Only the FP64 product emulated by the Ozaki scheme (MM_MODE_OZAKI) at
    n = m = p = --dgemm-size on full 53-bit uniform[-1,1) operands (seeds
    20/21), --ozaki-slices digit slices: rate, per-kernel device time and the
    library's FP64 check.  Prints one JSON line; also the profiling driver of
    the emulation's kernels."""
    import torch

    import paper_1306_6192_gb300 as mm
    import synth
    torch.cuda.set_device(0)
    mm.check_status(mm.mm_init(device=0), "mm_init")
    mm.check_status(mm.mm_ozaki_slices(args.ozaki_slices), "mm_ozaki_slices")
    n = args.dgemm_size
    A = torch.from_numpy(synth.uniform_pm1_f64(20, (n, n))).cuda()
    B = torch.from_numpy(synth.uniform_pm1_f64(21, (n, n))).cuda()
    C = torch.empty((n, n), dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    run = lambda: mm.check_status(mm.mm_gemm_async(n, n, n, A, B, C, mm.MM_F64, mm.MM_MODE_OZAKI,
                                                   stream), "ozaki")
    for _ in range(args.warmup):
        run()
    torch.cuda.synchronize()
    mm.mm_trace_reset()
    mm.mm_trace_enable(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        run()
    e1.record(stream)
    torch.cuda.synchronize()
    mm.mm_trace_enable(False)
    ms = e0.elapsed_time(e1) / args.steps
    kernels = {}
    for k in OZAKI_TRACE:
        _, cnt, kms = mm.mm_trace_read(k)
        if cnt:
            kernels[k] = kms / args.steps
    check = gpu_check(mm, n, n, n, A, B, C, mm.MM_F64)
    mm.mm_shutdown()
    print(json.dumps({"metric": "FP64 GEMM TFLOP/s (Ozaki scheme)", "value": 2.0 * n ** 3 / (ms * 1e-3) / 1e12,
                      "unit": "TFLOP/s", "n": n, "slices": args.ozaki_slices, "ms": ms,
                      "steps": args.steps, "kernels_ms": kernels, "check": check}))
    return 0


def run_stress_only(args):
    """Only the config-3 stress shapes (bench_stress).  Prints one JSON line."""
    import torch

    import paper_1306_6192_gb300 as mm
    torch.cuda.set_device(0)
    mm.check_status(mm.mm_init(device=0), "mm_init")
    stream = torch.cuda.Stream()
    peaks, _ = _peaks()
    out = bench_stress(mm, stream, peaks)
    mm.mm_shutdown()
    print(json.dumps({"metric": "stress shapes", "stress_shapes": out}))
    return 0 if "error" not in out else 1


def run_epilogue_only(args):
    """Only C = A.B - D at n^3 on the split path (default 4096): the product,
    the product then mm_add, and the subtraction fused into the product's
    epilogue (mm_gemm_axpby), 20 queued calls each, plus one synchronous
    fused call checked against the product minus D.  Prints one JSON line."""
    import torch

    import paper_1306_6192_gb300 as mm
    torch.cuda.set_device(0)
    mm.check_status(mm.mm_init(device=0), "mm_init")
    stream = torch.cuda.Stream()
    n = args.epilogue_size
    gen = torch.Generator(device="cuda")
    gen.manual_seed(3)
    A = torch.rand((n, n), device="cuda", generator=gen) * 2 - 1
    B = torch.rand((n, n), device="cuda", generator=gen) * 2 - 1
    D = torch.rand((n, n), device="cuda", generator=gen) * 2 - 1
    C = torch.empty((n, n), device="cuda")
    X = torch.empty((n, n), device="cuda")
    F32, X3 = mm.MM_F32, mm.MM_MODE_SPLIT_BF16X3
    ok = mm.check_status

    def queued(fn, k=20):
        fn()
        ok(mm.mm_sync(stream), "sync")
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    def two():
        ok(mm.mm_gemm_async(n, n, n, A, B, C, F32, X3, stream), "gemm")
        ok(mm.mm_add_async(n, n, 1.0, C, -1.0, D, C, F32, stream), "add")

    out = {"n": n,
           "gemm_ms": queued(lambda: ok(mm.mm_gemm_async(n, n, n, A, B, C, F32, X3, stream), "g")),
           "gemm_then_add_ms": queued(two),
           "fused_ms": queued(lambda: ok(mm.mm_gemm_axpby_async(n, n, n, 1.0, A, B, -1.0, D, C,
                                                                  F32, X3, stream), "f"))}
    ok(mm.mm_gemm(n, n, n, A, B, X, F32, X3), "gemm")
    ok(mm.mm_gemm_axpby(n, n, n, 1.0, A, B, -1.0, D, C, F32, X3), "axpby")
    out["fused_equals_product_minus_d"] = bool(torch.equal(C, X - D))
    mm.mm_shutdown()
    print(json.dumps({"metric": "fused epilogue", "epilogue": out}))
    return 0 if out["fused_equals_product_minus_d"] else 1


def run_serve_sweep(args):
    """Config-5 sweep: the Poisson replay at several fractions of the measured
    capacity, batched (2 streams, up to 256 per launch) against one request
    per launch on one stream, same arrivals.  Prints one JSON line."""
    import torch

    import paper_1306_6192_gb300 as mm
    torch.cuda.set_device(0)
    mm.check_status(mm.mm_init(device=0), "mm_init")
    f64_md = mm.MM_MODE_OZAKI if args.serve_f64 == "ozaki" else mm.MM_MODE_DGEMM
    rows = []
    cap = None
    for frac in args.serve_rates:
        row = {"rate_frac": frac}
        for name, st_, mb in (("batched", 2, 0), ("one_per_launch", 1, 1)):
            r = bench_serving(mm, args.serve_requests, frac, streams=st_, max_batch=mb,
                              capacity=cap, f64_mode=f64_md)
            cap = r["capacity_req_s"] if cap is None else cap
            row[name] = {k: r[k] for k in ("rate_req_s", "p50_ms", "p99_ms", "throughput_req_s",
                                           "tflops", "batches", "f32_split", "f64") if k in r}
        rows.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
    # the FP64 GPU check of every result, at 0.9 x capacity, on a shorter replay
    chk = bench_serving(mm, min(args.serve_requests, 5000), 0.9, streams=2, max_batch=0,
                        capacity=cap, f64_mode=f64_md, check=True)
    mm.mm_shutdown()
    print(json.dumps({"metric": "serving p50/p99 ms", "requests": args.serve_requests,
                      "capacity_req_s": cap, "mix": "dims log-uniform [64,4096], 20% FP64",
                      "f64_path": args.serve_f64, "sweep": rows,
                      "checked_replay": {k: chk[k] for k in ("requests", "f32_split", "f64")
                                         if k in chk}}))
    return 0


def run_mine(args):
    import numpy as np
    import torch

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_1306_6192_gb300 as mm
    import synth

    mm.check_status(mm.mm_init(device=local), "mm_init")
    n = args.size
    flops = 2.0 * n * n * n
    # every rank multiplies its own operands (independent problems)
    A = torch.from_numpy(synth.uniform_pm1(0 + 2 * rank, (n, n))).cuda()
    B = torch.from_numpy(synth.uniform_pm1(1 + 2 * rank, (n, n))).cuda()
    C = torch.empty((n, n), device="cuda")
    stream = torch.cuda.Stream()
    mode = {"split": mm.MM_MODE_SPLIT_BF16X3, "simt": mm.MM_MODE_SIMT}[args.mode]

    def step(md=mode, a=A, b=B, c=C, dt=mm.MM_F32, sz=None):
        sz = n if sz is None else sz
        st = mm.mm_gemm_async(sz, sz, sz, a, b, c, dt, md, stream)
        if st != mm.MM_OK:
            raise mm.MMError(st, "mm_gemm_async")

    def barrier():
        if dist is not None:
            dist.barrier()

    def timed(fn, steps, warmup, trace=False):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        mm.check_status(mm.mm_sync(stream), "warmup")
        barrier()
        torch.cuda.synchronize()
        if trace:
            mm.mm_trace_reset()
            mm.mm_trace_enable(True)
        l0 = mm.mm_launch_count()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        launches = mm.mm_launch_count() - l0
        barrier()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        if trace:
            mm.mm_trace_enable(False)
        mm.check_status(mm.mm_sync(stream), "timed")
        return max_over_ranks(ms, dist, "cuda"), launches

    with Clocks(local) as clk:
        ms, launches = timed(step, args.steps, args.warmup, trace=True)
    clocks = clk.summary()
    clocks["window"] = "the timed region"
    per_kernel = {}
    for k in ("split_scale", "split_pack", "split_verify", "split_fix", "split_tc", "simt_f32"):
        st, cnt, kms = mm.mm_trace_read(k)
        if cnt:
            per_kernel[k] = {"launches": cnt, "avg_ms": kms / cnt}
    mm.mm_trace_reset()
    ms_step = ms / args.steps
    value = whole_job_rate(flops, world, ms_step) / 1e12

    peaks, peak_src = _peaks()
    line = {
        "metric": "GEMM TFLOP/s", "value": value, "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16x3->f32" if args.mode == "split" else "f32", "data": "synthetic",
        "path": "split-BF16x3 tcgen05" if args.mode == "split" else "SIMT FP32",
        "config": workload_config(n, world),
        "gpu_launches": launches, "clocks": clocks, "kernels": per_kernel,
    }
    if args.mode == "split" and "split_tc" in per_kernel:
        avg = per_kernel["split_tc"]["avg_ms"]
        # burst peak for a timed region under a second, sustained beyond
        kind = "sustained" if ms > 1000.0 else "burst"
        peak = peaks.get("bf16_tflops_sustained" if kind == "sustained" else "bf16_tflops",
                         1700.0) / 3.0
        ach = flops / (avg * 1e-3) / 1e12
        line["roofline"] = {
            "bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
            "frac": ach / peak, "traffic": _traffic_from_profiles("tc_gemm_split_8192.txt"),
            "kernel": "split_tc",
            "peak_note": "%s %s BF16 dense / 3 (three BF16 products per useful FMA)" % (
                peak_src, kind),
        }

    if rank == 0 and not args.quick:
        # other paths at the same size, for the split/SIMT ratio and FP64 rate
        extra = {}
        if args.mode == "split":
            ms_s, _ = timed(lambda: step(mm.MM_MODE_SIMT), max(2, args.steps // 4), 1)
            extra["simt_f32_tflops"] = flops / (ms_s / max(2, args.steps // 4) * 1e-3) / 1e12
            extra["split_over_simt"] = value / world / extra["simt_f32_tflops"]
            # the CUDA cores' measured FFMA rate right after (the same clock):
            # the SIMT kernel's roofline
            st32, f32 = mm.mm_measure_fma_peak(mm.MM_F32, 4096)
            if st32 == mm.MM_OK and f32 > 0:
                extra["ffma_peak_tflops"] = f32 / 1e12
                extra["simt_frac_of_measured_ffma"] = extra["simt_f32_tflops"] / (f32 / 1e12)
        nd = args.dgemm_size
        A64 = A[:nd, :nd].double().contiguous()
        B64 = B[:nd, :nd].double().contiguous()
        C64 = torch.empty((nd, nd), device="cuda", dtype=torch.float64)
        f64 = lambda: mm.mm_gemm_async(nd, nd, nd, A64, B64, C64, mm.MM_F64, mm.MM_MODE_DGEMM,
                                       stream)
        ms_d, _ = timed(f64, 2, 1)
        extra["dgemm_f64_tflops"] = 2.0 * nd ** 3 / (ms_d / 2 * 1e-3) / 1e12
        extra["dgemm_size"] = nd
        # the CUDA cores' measured DFMA rate right after the DGEMM timing (at
        # the same clock): the DGEMM roofline
        st64, f64r = mm.mm_measure_fma_peak(mm.MM_F64, 256)
        if st64 == mm.MM_OK and f64r > 0:
            extra["dfma_peak_tflops"] = f64r / 1e12
            extra["dgemm_frac_of_measured_dfma"] = extra["dgemm_f64_tflops"] / (f64r / 1e12)
        extra["dgemm_check"] = gpu_check(mm, nd, nd, nd, A64, B64, C64, mm.MM_F64)
        # FP64 emulated on the e4m3 tensor cores (Ozaki scheme, default slices)
        # on full 53-bit FP64 operands of the same size
        A64 = torch.from_numpy(synth.uniform_pm1_f64(20, (nd, nd))).cuda()
        B64 = torch.from_numpy(synth.uniform_pm1_f64(21, (nd, nd))).cuda()
        oz = lambda: mm.check_status(mm.mm_gemm_async(nd, nd, nd, A64, B64, C64, mm.MM_F64,
                                                      mm.MM_MODE_OZAKI, stream), "ozaki")
        ms_o, _ = timed(oz, 5, 2, trace=True)
        extra["ozaki_f64_tflops"] = 2.0 * nd ** 3 / (ms_o / 5 * 1e-3) / 1e12
        extra["ozaki_over_dgemm"] = extra["ozaki_f64_tflops"] / extra["dgemm_f64_tflops"]
        extra["ozaki_kernels_ms"] = {}
        for k in OZAKI_TRACE:
            _, cnt, kms = mm.mm_trace_read(k)
            if cnt:
                extra["ozaki_kernels_ms"][k] = kms / 5
        mm.mm_trace_reset()
        extra["ozaki_check"] = gpu_check(mm, nd, nd, nd, A64, B64, C64, mm.MM_F64)
        del A64, B64, C64
        # FP8 e4m3 at the same size: rate and measured error (reported only)
        ms_8, _ = timed(lambda: step(mm.MM_MODE_FP8), max(2, args.steps // 4), 1, trace=True)
        extra["fp8_tflops"] = flops / (ms_8 / max(2, args.steps // 4) * 1e-3) / 1e12
        _, k8, t8 = mm.mm_trace_read("fp8_tc")
        _, _, tb = mm.mm_trace_read("fp8_blk")
        if k8:
            # its tensor-core kernels (the 128 x 256 one when every tile keeps
            # one exponent along K, else the blockwise one; the other returns at
            # once) against the nominal FP8 rate: the measured burst BF16 peak x
            # 2 (FP8 / BF16 dense ratio)
            extra["fp8_tc_tflops"] = flops / ((t8 + tb) / k8 * 1e-3) / 1e12
            extra["fp8_tc_frac"] = extra["fp8_tc_tflops"] / (2.0 * peaks.get("bf16_tflops", 1941.7))
        mm.mm_trace_reset()
        extra["fp8_check"] = gpu_check(mm, n, n, n, A, B, C, mm.MM_F32)
        # accuracy of the headline product, FP64 check on the GPU
        step()
        mm.check_status(mm.mm_sync(stream), "split")
        extra["split_check"] = gpu_check(mm, n, n, n, A, B, C, mm.MM_F32)
        extra["tolerance_f32"] = 1e-6 * n ** 0.5
        # the other square sizes of the workload (device time, same stream)
        sizes = {}
        for sz in (1024, 2048, 4096):
            a, b, c = A[:sz, :sz].contiguous(), B[:sz, :sz].contiguous(), C.view(-1)[:sz * sz]
            reps = 20
            ms_z, _ = timed(lambda: step(mode, a, b, c, sz=sz), reps, 3)
            ms_y, _ = timed(lambda: step(mm.MM_MODE_SIMT, a, b, c, sz=sz), 5, 1)
            sizes[str(sz)] = {"split_tflops": 2.0 * sz ** 3 / (ms_z / reps * 1e-3) / 1e12,
                              "simt_tflops": 2.0 * sz ** 3 / (ms_y / 5 * 1e-3) / 1e12}
        extra["square_sizes"] = sizes
        line["paths"] = extra
        line["paper_workloads_4096"] = bench_paper_workloads(mm, stream, peaks)
        line["stress_shapes"] = bench_stress(mm, stream, peaks)
        line["grouped"] = bench_grouped(mm, stream, max(3, args.steps // 20))
        cap = None
        serving = {}
        for name, st_, mb in (("batched", 2, 0), ("one_per_launch", 1, 1)):
            r = bench_serving(mm, args.serve_requests, 0.9, streams=st_, max_batch=mb,
                              capacity=cap)
            cap = r["capacity_req_s"] if cap is None else cap
            serving[name] = r
        # the same arrivals with the FP64 requests on the emulated path
        serving["batched_ozaki_f64"] = bench_serving(mm, args.serve_requests, 0.9, streams=2,
                                                     max_batch=0, capacity=None,
                                                     f64_mode=mm.MM_MODE_OZAKI)
        line["serving"] = serving

        # end to end: mm_gemm with pinned host operands, copies inside the timing
        Ah = A.cpu().pin_memory()
        Bh = B.cpu().pin_memory()
        Ch = torch.empty((n, n), dtype=torch.float32).pin_memory()
        torch.cuda.synchronize()
        mm.check_status(mm.mm_gemm(n, n, n, Ah, Bh, Ch, mm.MM_F32, mode), "e2e warmup")
        k = max(2, args.steps // 4)
        t0 = time.perf_counter()
        for _ in range(k):
            mm.check_status(mm.mm_gemm(n, n, n, Ah, Bh, Ch, mm.MM_F32, mode), "e2e")
        t_e2e = (time.perf_counter() - t0) / k
        line["e2e"] = {"value": flops / t_e2e / 1e12, "unit": "TFLOP/s",
                       "h2d_bytes_per_step": 2 * n * n * 4, "d2h_bytes_per_step": n * n * 4}
        del Ah, Bh, Ch

    # the headline step again, untimed, for 1.5 s with the clocks sampled: the
    # timed region alone can be shorter than a few 50 ms sampling intervals.
    # Run last, so that the power-capped clock of a sustained run does not
    # carry over into the other legs.
    with Clocks(local) as clk2:
        t_end = time.perf_counter() + 1.5
        while time.perf_counter() < t_end:
            for _ in range(10):
                step()
            torch.cuda.synchronize()
    line["clocks_steady"] = dict(clk2.summary(), window="1.5 s of the headline step, after the other legs")

    if rank == 0 and not args.no_cpu_baseline and not args.quick:
        rate, cores, rows, t = oracle_sample_rate(n)
        line["cpu_baseline"] = {"value": rate, "unit": "TFLOP/s", "cores": cores,
                                "kind": "oracle",
                                "sample": "%d of %d rows of C, FP64, %.1f s" % (rows, n, t)}
    mm.mm_shutdown()
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_shard(args):
    """One product split by row blocks over the ranks (strong scaling): rank r
    multiplies its rows [r0, r1) of A by the replicated B into its rows of C
    (paper_1306_6192_gb300.shard), with no collective inside the timed
    region; an NCCL all-gather of the C blocks is timed afterwards and
    reported on its own."""
    import torch

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_1306_6192_gb300 as mm
    from paper_1306_6192_gb300 import shard
    import synth

    mm.check_status(mm.mm_init(device=local), "mm_init")
    n = args.size
    r0, r1 = shard.local_block(n, rank, world)
    A = torch.from_numpy(synth.uniform_pm1(0, (n, n))[r0:r1]).cuda()  # this rank's rows
    B = torch.from_numpy(synth.uniform_pm1(1, (n, n))).cuda()         # replicated
    C = torch.empty((r1 - r0, n), device="cuda")
    stream = torch.cuda.Stream()
    md = {"split": mm.MM_MODE_SPLIT_BF16X3, "simt": mm.MM_MODE_SIMT}[args.mode]

    def step():
        if r1 > r0:
            mm.check_status(mm.mm_gemm_async(r1 - r0, n, n, A, B, C, mm.MM_F32, md, stream),
                            "shard")

    for _ in range(args.warmup):
        step()
    mm.check_status(mm.mm_sync(stream), "warmup")
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = mm.mm_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    launches = mm.mm_launch_count() - l0
    mm.check_status(mm.mm_sync(stream), "timed")
    ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda") / args.steps
    gather_ms = None
    if dist is not None:
        rows = max(b1 - b0 for b0, b1 in shard.row_blocks(n, world))
        buf = torch.zeros((rows, n), device="cuda")
        buf[: r1 - r0] = C
        parts = [torch.empty_like(buf) for _ in range(world)]
        dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dist.all_gather(parts, buf)
        torch.cuda.synchronize()
        gather_ms = max_over_ranks((time.perf_counter() - t0) * 1e3, dist, "cuda")
    flops = 2.0 * n * n * n
    line = {
        "metric": "GEMM TFLOP/s", "value": flops / (ms * 1e-3) / 1e12, "unit": "TFLOP/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
        "dtype": "bf16x3->f32" if args.mode == "split" else "f32", "data": "synthetic",
        "path": "row blocks of one product, split-BF16x3 tcgen05 per rank",
        "config": dict(workload_config(n, world), parallelism="row blocks x%d" % world,
                       rows_per_rank=[b1 - b0 for b0, b1 in shard.row_blocks(n, world)]),
        "gpu_launches": launches, "clocks": clk.summary(),
        "gather_ms": gather_ms,
    }
    mm.mm_shutdown()
    if dist is not None:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["mine", "reference"], default="mine")
    ap.add_argument("--size", type=int, default=N_DEFAULT)
    ap.add_argument("--mode", choices=["split", "simt"], default="split")
    ap.add_argument("--dgemm-size", type=int, default=4096)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true", help="headline step only")
    ap.add_argument("--serve-requests", type=int, default=1500)
    ap.add_argument("--serve-sweep", action="store_true",
                    help="only the serving rate sweep (config 5)")
    ap.add_argument("--serve-rates", type=float, nargs="*",
                    default=[0.1, 0.25, 0.5, 0.75, 0.9, 1.0, 1.1])
    ap.add_argument("--grouped-only", action="store_true",
                    help="only the grouped leg (config 4), --steps grouped launches")
    ap.add_argument("--grouped-count", type=int, default=4096)
    ap.add_argument("--ozaki-only", action="store_true",
                    help="only the FP64 product emulated by the Ozaki scheme")
    ap.add_argument("--ozaki-slices", type=int, default=12)
    ap.add_argument("--fp8-only", action="store_true",
                    help="only the FP8 e4m3 product at --size")
    ap.add_argument("--stress-only", action="store_true", help="only the config-3 stress shapes")
    ap.add_argument("--epilogue-only", action="store_true",
                    help="only C = A.B - D, fused into the product's epilogue and as two calls")
    ap.add_argument("--epilogue-size", type=int, default=4096)
    ap.add_argument("--serve-f64", choices=["dgemm", "ozaki"], default="dgemm",
                    help="path of the serving mix's FP64 requests")
    ap.add_argument("--shard", choices=["none", "rows"], default="none",
                    help="rows: one product split by row blocks over the ranks (strong scaling)")
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "mine":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.serve_sweep:
        return run_serve_sweep(args)
    if args.grouped_only:
        return run_grouped_only(args)
    if args.ozaki_only:
        return run_ozaki_only(args)
    if args.stress_only:
        return run_stress_only(args)
    if args.epilogue_only:
        return run_epilogue_only(args)
    if args.fp8_only:
        return run_fp8_only(args)
    if args.shard == "rows":
        return run_shard(args)
    return run_mine(args)


if __name__ == "__main__":
    sys.exit(main())
