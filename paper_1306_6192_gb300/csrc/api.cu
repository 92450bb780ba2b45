// C ABI of the library (include/mm.h): context, scratch memory, dispatch to
// the kernels, tracing.  The serving loop lives in serve.cu, the autotuner
// table in tune.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <map>

#include "ctx.h"

namespace mm {

Ctx g_ctx;
std::mutex g_api_mutex;

// ---------------------------------------------------------------- errors
mm_status from_cuda(cudaError_t e) {
  switch (e) {
    case cudaSuccess: return MM_OK;
    case cudaErrorMemoryAllocation: return MM_ENOMEM;
    case cudaErrorInvalidValue: return MM_EINVAL;
    case cudaErrorNotSupported: return MM_EUNSUPPORTED;
    default: return MM_ECUDA;
  }
}

// A sticky error (illegal address, launch failure ...) loses the context: the
// library then refuses further work.
mm_status note_cuda(cudaError_t e) {
  if (e == cudaSuccess) return MM_OK;
  cudaError_t last = cudaGetLastError();
  (void)last;
  cudaError_t probe = cudaDeviceSynchronize();
  if (probe != cudaSuccess && probe != cudaErrorNotReady) g_ctx.sticky = true;
  return from_cuda(e);
}

int sm_count() { return g_ctx.sms > 0 ? g_ctx.sms : 148; }

// ---------------------------------------------------------------- scratch
cudaError_t Scratch::reserve(size_t need, cudaStream_t s) {
  if (need <= bytes) return cudaSuccess;
  // grow by at least a quarter of the old size, so that a run of slightly
  // larger requests does not pay a synchronisation and a reallocation each
  const size_t old = bytes;
  if (ptr) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
  }
  size_t want = std::max(need, old + old / 4);
  want = (want + (1u << 20) - 1) & ~(size_t)((1u << 20) - 1);
  cudaError_t e = cudaMalloc(&ptr, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    e = cudaMalloc(&ptr, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      ptr = nullptr;
      return cudaErrorMemoryAllocation;
    }
    want = need;
  }
  bytes = want;
  return cudaSuccess;
}

void Scratch::release() {
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
  bytes = 0;
  stage.release();
}

cudaError_t HostStage::copy_to_device(void *dst, const void *src, size_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int k = next;
  next = (next + 1) % kSlots;
  if (pending[k]) {
    cudaError_t e = cudaEventSynchronize(ev[k]);  // that slot's copy has run
    if (e != cudaSuccess) return e;
    pending[k] = false;
  }
  if (n > bytes[k]) {
    if (ptr[k]) cudaFreeHost(ptr[k]);
    ptr[k] = nullptr;
    bytes[k] = 0;
    const size_t want = std::max(n, (size_t)64 << 10);
    if (cudaMallocHost(&ptr[k], want) != cudaSuccess) {
      cudaGetLastError();
      ptr[k] = nullptr;
      return cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, s);  // pageable fallback
    }
    bytes[k] = want;
  }
  if (!ev[k] && cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    ev[k] = nullptr;
    return cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, s);
  }
  std::memcpy(ptr[k], src, n);
  cudaError_t e = cudaMemcpyAsync(dst, ptr[k], n, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  e = cudaEventRecord(ev[k], s);
  pending[k] = e == cudaSuccess;
  return e;
}

void HostStage::release() {
  for (int k = 0; k < kSlots; k++) {
    if (pending[k] && ev[k]) cudaEventSynchronize(ev[k]);
    if (ptr[k]) cudaFreeHost(ptr[k]);
    if (ev[k]) cudaEventDestroy(ev[k]);
    ptr[k] = nullptr;
    ev[k] = nullptr;
    bytes[k] = 0;
    pending[k] = false;
  }
  next = 0;
}

// ---------------------------------------------------------------- tracing
namespace {
struct TraceRec {
  const char *name;
  cudaEvent_t a, b;
};
std::mutex g_trace_mu;
bool g_trace_on = false;
std::vector<TraceRec> g_trace_open;   // begun, waiting for end
std::vector<TraceRec> g_trace_done;
std::vector<cudaEvent_t> g_event_pool;
std::atomic<int64_t> g_launches{0};

cudaEvent_t take_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

void trace_begin(const char *name, cudaStream_t s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  std::lock_guard<std::mutex> lk(g_trace_mu);
  if (!g_trace_on) return;
  TraceRec r{name, take_event(), take_event()};
  cudaEventRecord(r.a, s);
  g_trace_open.push_back(r);
}

void trace_end(const char *name, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_trace_mu);
  if (!g_trace_on) return;
  for (size_t i = g_trace_open.size(); i-- > 0;) {
    if (g_trace_open[i].name == name) {
      TraceRec r = g_trace_open[i];
      g_trace_open.erase(g_trace_open.begin() + (long)i);
      cudaEventRecord(r.b, s);
      g_trace_done.push_back(r);
      return;
    }
  }
}

void trace_clear() {
  std::lock_guard<std::mutex> lk(g_trace_mu);
  for (auto &r : g_trace_done) {
    g_event_pool.push_back(r.a);
    g_event_pool.push_back(r.b);
  }
  g_trace_done.clear();
}

static void trace_destroy() {
  trace_clear();
  std::lock_guard<std::mutex> lk(g_trace_mu);
  for (auto &r : g_trace_open) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  g_trace_open.clear();
  for (auto e : g_event_pool) cudaEventDestroy(e);
  g_event_pool.clear();
  g_trace_on = false;
}

// ---------------------------------------------------------------- pointers
// Classifies a pointer: 1 = device-accessible (device or managed memory of
// the current device), 0 = host memory (pinned or pageable), -1 = invalid.
int pointer_kind(const void *p) {
  if (!p) return -1;
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  switch (at.type) {
    case cudaMemoryTypeDevice:
    case cudaMemoryTypeManaged: return 1;
    default: return 0;
  }
}

// ---------------------------------------------------------------- dispatch
static mm_mode resolve_mode(mm_dtype dt, mm_mode mode) {
  if (mode == MM_MODE_AUTO) return dt == MM_F64 ? MM_MODE_DGEMM : MM_MODE_SPLIT_BF16X3;
  return mode;
}

mm_status validate(int64_t n, int64_t m, int64_t p, mm_dtype dt, mm_mode mode) {
  if (n < 0 || m < 0 || p < 0) return MM_EINVAL;
  if (dt != MM_F32 && dt != MM_F64) return MM_EINVAL;
  if ((int)mode < 0 || (int)mode > (int)MM_MODE_SPLIT_BF16X6) return MM_EINVAL;
  const mm_mode md = resolve_mode(dt, mode);
  const bool f64_mode = md == MM_MODE_DGEMM || md == MM_MODE_OZAKI;
  if (dt == MM_F64 && !f64_mode) return MM_EUNSUPPORTED;
  if (dt == MM_F32 && f64_mode) return MM_EUNSUPPORTED;
  // 32-bit tile bookkeeping of the kernels
  if (n > (int64_t)1 << 31 || m > (int64_t)1 << 31 || p > (int64_t)1 << 31) return MM_EINVAL;
  return MM_OK;
}

// The epilogue C = alpha (A.B) + beta D as a pass of its own after the
// product, for the paths whose kernels have no slack for it: the product goes
// to C (or to library scratch where D is C), then one elementwise kernel with
// the fused form's arithmetic (the same bits).
template <typename Run>
static mm_status product_then_epilogue(int64_t n, int64_t p, void *C, mm_dtype dt, const Epi &epi,
                                       cudaStream_t s, Run run) {
  const bool two = dt == MM_F32 ? (float)epi.beta != 0.0f : epi.beta != 0.0;
  void *X = C;
  if (two && epi.D == C) {
    cudaError_t e = g_ctx.epi_ws.reserve((size_t)(n * p) * (dt == MM_F64 ? 8 : 4), s);
    if (e != cudaSuccess) return note_cuda(e);
    X = g_ctx.epi_ws.ptr;
  }
  mm_status st = run(X);
  if (st != MM_OK) return st;
  if (two) return enqueue_add(n, p, epi.alpha, X, epi.beta, epi.D, C, dt, s);
  const bool unit = dt == MM_F32 ? (float)epi.alpha == 1.0f : epi.alpha == 1.0;
  return unit ? MM_OK : enqueue_scale(n * p, epi.alpha, C, C, dt, s);
}

// Queues C = A.B (device pointers) on stream s.
mm_status enqueue_gemm(int64_t n, int64_t m, int64_t p, const void *A, const void *B, void *C,
                       mm_dtype dt, mm_mode mode, cudaStream_t s, const Epi *epi) {
  const mm_mode md = resolve_mode(dt, mode);
  if (n == 0 || p == 0) return MM_OK;
  if (m == 0) {
    // alpha (A.B) = 0: C = beta D
    if (epi) return enqueue_scale(n * p, epi->beta, epi->D, C, dt, s);
    const size_t es = dt == MM_F64 ? 8 : 4;
    return note_cuda(cudaMemsetAsync(C, 0, (size_t)(n * p) * es, s));
  }
  switch (md) {
    case MM_MODE_SIMT:
    case MM_MODE_DGEMM: {
      // products with few output tiles: K slices and a fixed-order sum
      const bool f64 = md == MM_MODE_DGEMM;
      const SimtPlan pl = simt_plan(f64, n, m, p);
      if (pl.S >= 1) {
        void *part = nullptr;
        if (pl.S > 1) {
          cudaError_t e = g_ctx.simt_ws.reserve(simt_scratch_bytes(f64, n, m, p), s);
          if (e != cudaSuccess) return note_cuda(e);
          part = g_ctx.simt_ws.ptr;
        }
        return note_cuda(f64 ? launch_simt_splitk_f64(n, m, p, (const double *)A, (const double *)B,
                                                      (double *)C, (double *)part, pl, s, nullptr,
                                                      epi)
                             : launch_simt_splitk_f32(n, m, p, (const float *)A, (const float *)B,
                                                      (float *)C, (float *)part, pl, s, epi));
      }
      return note_cuda(f64 ? launch_simt_f64(n, m, p, (const double *)A, (const double *)B,
                                             (double *)C, s, nullptr, epi)
                           : launch_simt_f32(n, m, p, (const float *)A, (const float *)B,
                                             (float *)C, s, epi));
    }
    case MM_MODE_SPLIT_BF16X3:
    case MM_MODE_SPLIT_BF16X6: {
      // two or three parts by m (x3), three parts (x6); products with few
      // output tiles run as one fused split-K launch
      const TcKind kind = split_kind_of(md, m);
      const FusedPlan fpl = fused_plan(n, m, p, kind);
      if (fpl.S > 0 && fused_operands_ok(static_cast<const float *>(A),
                                         static_cast<const float *>(B), m, p)) {
        return run_fused(g_ctx.fused_ws, n, m, p, static_cast<const float *>(A),
                         static_cast<const float *>(B), static_cast<float *>(C), kind, fpl, s, epi);
      }
      mm_problem q{n, m, p, A, B, C};
      return run_split(g_ctx.split_ws, &q, 1, s, nullptr, md == MM_MODE_SPLIT_BF16X6, epi);
    }
    case MM_MODE_FP8: {
      // the e4m3 tiles' MMAs take about as long as their stores, so the
      // epilogue runs as a pass of its own (measured faster than fused)
      auto run = [&](void *X) {
        mm_problem q{n, m, p, A, B, X};
        return run_fp8(g_ctx.fp8_ws, &q, 1, s);
      };
      return epi ? product_then_epilogue(n, p, C, dt, *epi, s, run) : run(C);
    }
    case MM_MODE_OZAKI:
      return run_ozaki(g_ctx.ozaki_ws, n, m, p, (const double *)A, (const double *)B, (double *)C,
                       g_ctx.ozaki_slices, g_ctx.ozaki_gate != 0, s, epi);
    default: return MM_EINVAL;
  }
}

mm_status check_device_flag(cudaStream_t s) {
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return note_cuda(e);
  int flag = 0;
  e = cudaMemcpy(&flag, g_ctx.d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return note_cuda(e);
  if (flag != 0) {
    cudaMemset(g_ctx.d_err, 0, sizeof(int));
    g_ctx.fused_zero_ptr = nullptr;  // an aborted fused launch may leave counters set
    return MM_ETIMEOUT;
  }
  return MM_OK;
}

}  // namespace mm

using namespace mm;

#define MM_REQUIRE_INIT()                    \
  do {                                       \
    if (!g_ctx.inited) return MM_ENOTINIT;   \
    if (g_ctx.sticky) return MM_ECUDA;       \
  } while (0)

extern "C" {

const char *mm_strerror(mm_status s) {
  switch (s) {
    case MM_OK: return "ok";
    case MM_EINVAL: return "invalid argument";
    case MM_ENOMEM: return "out of memory";
    case MM_EBUDGET: return "request exceeds the HBM budget";
    case MM_EBUSY: return "already initialised";
    case MM_ENOTFOUND: return "unknown request id";
    case MM_EPENDING: return "request pending";
    case MM_ETIMEOUT: return "bounded wait timed out";
    case MM_ECUDA: return "CUDA error";
    case MM_ENOTINIT: return "library not initialised";
    case MM_EUNSUPPORTED: return "unsupported dtype/mode or device";
    case MM_ECANCELLED: return "request cancelled";
    case MM_ESCRATCH: return "product too large for the fixed scratch array";
  }
  return "unknown status";
}

mm_status mm_init(const mm_opts *opts) {
  std::lock_guard<std::mutex> lk(g_api_mutex);
  if (g_ctx.inited) return MM_EBUSY;
  mm_opts o;
  std::memset(&o, 0, sizeof(o));
  o.device = -1;
  if (opts) o = *opts;
  if (o.hbm_budget_bytes == 0) o.hbm_budget_bytes = (size_t)40 << 30;
  if (o.n_streams <= 0) o.n_streams = 2;
  if (o.n_streams > 8) o.n_streams = 8;
  int dev = 0;
  cudaError_t e;
  if (o.device >= 0) {
    e = cudaSetDevice(o.device);
    if (e != cudaSuccess) return from_cuda(e);
  }
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return from_cuda(e);
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, dev);
  if (e != cudaSuccess) return from_cuda(e);
  // The kernels are built for sm_103a only.
  if (prop.major != 10 || prop.minor != 3) return MM_EUNSUPPORTED;
  g_ctx.device = dev;
  g_ctx.sms = prop.multiProcessorCount;
  g_ctx.opts = o;
  e = cudaStreamCreateWithFlags(&g_ctx.stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return from_cuda(e);
  e = cudaMalloc(&g_ctx.d_err, 256);
  if (e != cudaSuccess) {
    cudaStreamDestroy(g_ctx.stream);
    return from_cuda(e);
  }
  bool ok = cudaStreamCreateWithFlags(&g_ctx.h2d, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&g_ctx.d2h, cudaStreamNonBlocking) == cudaSuccess;
  for (int c = 0; c <= Ctx::kMaxChunks && ok; c++)
    ok = cudaEventCreateWithFlags(&g_ctx.ev_in[c], cudaEventDisableTiming) == cudaSuccess;
  for (int c = 0; c < Ctx::kMaxChunks && ok; c++)
    ok = cudaEventCreateWithFlags(&g_ctx.ev_out[c], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&g_ctx.ev_prep[c], cudaEventDisableTiming) == cudaSuccess;
  for (auto &ts : g_ctx.tc_streams)
    ok = ok && cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking) == cudaSuccess;
  if (!ok) return MM_ECUDA;
  cudaMemset(g_ctx.d_err, 0, 256);
  tune_reset_defaults();
  if (o.tune_table) {
    mm_status st = tune_load_file(o.tune_table);
    if (st != MM_OK) {
      cudaFree(g_ctx.d_err);
      cudaStreamDestroy(g_ctx.stream);
      return st;
    }
  }
  g_ctx.sticky = false;
  g_ctx.inited = true;
  mm_status st = serve_start();
  if (st != MM_OK) {
    g_ctx.inited = false;
    cudaFree(g_ctx.d_err);
    cudaStreamDestroy(g_ctx.stream);
    return st;
  }
  return MM_OK;
}

mm_status mm_shutdown(void) {
  std::lock_guard<std::mutex> lk(g_api_mutex);
  if (!g_ctx.inited) return MM_OK;
  serve_stop();
  cudaStreamSynchronize(g_ctx.stream);
  g_ctx.split_ws.release();
  g_ctx.fp8_ws.release();
  g_ctx.stage_ws.release();
  g_ctx.check_ws.release();
  g_ctx.cplx_ws.release();
  g_ctx.ozaki_ws.release();
  g_ctx.fused_ws.release();
  g_ctx.simt_ws.release();
  g_ctx.epi_ws.release();
  g_ctx.fused_zero_ptr = nullptr;
  g_ctx.fused_zeroed = 0;
  g_ctx.ozaki_slices = kOzakiDefaultSlices;
  g_ctx.ozaki_gate = 1;
  if (g_ctx.d_err) cudaFree(g_ctx.d_err);
  g_ctx.d_err = nullptr;
  trace_destroy();
  for (auto &ev : g_ctx.ev_in)
    if (ev) cudaEventDestroy(ev), ev = nullptr;
  for (auto &ev : g_ctx.ev_out)
    if (ev) cudaEventDestroy(ev), ev = nullptr;
  for (auto &ev : g_ctx.ev_prep)
    if (ev) cudaEventDestroy(ev), ev = nullptr;
  for (auto &ts : g_ctx.tc_streams)
    if (ts) cudaStreamDestroy(ts), ts = nullptr;
  if (g_ctx.h2d) cudaStreamDestroy(g_ctx.h2d);
  if (g_ctx.d2h) cudaStreamDestroy(g_ctx.d2h);
  g_ctx.h2d = g_ctx.d2h = nullptr;
  cudaStreamDestroy(g_ctx.stream);
  g_ctx.stream = nullptr;
  g_ctx.inited = false;
  return MM_OK;
}

mm_status mm_ozaki_slices(int slices) {
  std::lock_guard<std::mutex> lk(g_api_mutex);
  if (!g_ctx.inited) return MM_ENOTINIT;
  if (slices < kOzakiMinSlices || slices > kOzakiMaxSlices) return MM_EINVAL;
  g_ctx.ozaki_slices = slices;
  return MM_OK;
}

mm_status mm_ozaki_gate(int on) {
  std::lock_guard<std::mutex> lk(g_api_mutex);
  if (!g_ctx.inited) return MM_ENOTINIT;
  if (on != 0 && on != 1) return MM_EINVAL;
  g_ctx.ozaki_gate = on;
  return MM_OK;
}

mm_status mm_gemm_async(int64_t n, int64_t m, int64_t p, const void *A, const void *B, void *C,
                        mm_dtype dt, mm_mode mode, void *stream) {
  MM_REQUIRE_INIT();
  mm_status st = validate(n, m, p, dt, mode);
  if (st != MM_OK) return st;
  if (n == 0 || p == 0) return MM_OK;
  if (!C || (m > 0 && (!A || !B))) return MM_EINVAL;
  if (pointer_kind(C) != 1 || (m > 0 && (pointer_kind(A) != 1 || pointer_kind(B) != 1)))
    return MM_EINVAL;
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : g_ctx.stream;
  std::lock_guard<std::mutex> lk(g_api_mutex);
  return enqueue_gemm(n, m, p, A, B, C, dt, mode, s);
}

// C = alpha (A.B) + beta D on device pointers: checks, then the product with
// its epilogue, or C = beta D where the product has no terms (alpha = 0 or
// m = 0: A and B are not read).
static mm_status enqueue_axpby(int64_t n, int64_t m, int64_t p, double alpha, const void *A,
                               const void *B, double beta, const void *D, void *C, mm_dtype dt,
                               mm_mode mode, cudaStream_t s) {
  mm_status st = validate(n, m, p, dt, mode);
  if (st != MM_OK) return st;
  if (n == 0 || p == 0) return MM_OK;
  const bool terms = m > 0 && alpha != 0.0;
  if (!C || pointer_kind(C) != 1) return MM_EINVAL;
  if (terms && (!A || !B || pointer_kind(A) != 1 || pointer_kind(B) != 1)) return MM_EINVAL;
  if (beta != 0.0) {
    if (!D || pointer_kind(D) != 1) return MM_EINVAL;
    // D is C itself or apart from it
    const size_t bytes = (size_t)(n * p) * (dt == MM_F64 ? 8 : 4);
    const uintptr_t d0 = reinterpret_cast<uintptr_t>(D), c0 = reinterpret_cast<uintptr_t>(C);
    if (d0 != c0 && d0 < c0 + bytes && c0 < d0 + bytes) return MM_EINVAL;
  }
  const Epi epi{alpha, beta, beta != 0.0 ? D : nullptr};
  if (!terms) return enqueue_scale(n * p, beta, epi.D, C, dt, s);
  return enqueue_gemm(n, m, p, A, B, C, dt, mode, s, &epi);
}

mm_status mm_gemm_axpby_async(int64_t n, int64_t m, int64_t p, double alpha, const void *A,
                              const void *B, double beta, const void *D, void *C, mm_dtype dt,
                              mm_mode mode, void *stream) {
  MM_REQUIRE_INIT();
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : g_ctx.stream;
  std::lock_guard<std::mutex> lk(g_api_mutex);
  return enqueue_axpby(n, m, p, alpha, A, B, beta, D, C, dt, mode, s);
}

mm_status mm_gemm_axpby(int64_t n, int64_t m, int64_t p, double alpha, const void *A,
                        const void *B, double beta, const void *D, void *C, mm_dtype dt,
                        mm_mode mode) {
  MM_REQUIRE_INIT();
  mm_status st = validate(n, m, p, dt, mode);
  if (st != MM_OK) return st;
  if (n == 0 || p == 0) return MM_OK;
  const bool terms = m > 0 && alpha != 0.0, with_d = beta != 0.0;
  if (!C || (terms && (!A || !B)) || (with_d && !D)) return MM_EINVAL;
  std::lock_guard<std::mutex> lk(g_api_mutex);
  cudaStream_t s = g_ctx.stream;
  const bool dev_c = pointer_kind(C) == 1;
  const bool dev_a = !terms || pointer_kind(A) == 1;
  const bool dev_b = !terms || pointer_kind(B) == 1;
  const bool dev_d = !with_d || pointer_kind(D) == 1;
  if (!(dev_a && dev_b && dev_c && dev_d)) {
    // Host operands: staged through library buffers on the library stream,
    // as mm_gemm does; D and C are checked for overlap as host ranges
    const size_t es = dt == MM_F64 ? 8 : 4;
    const size_t ba = terms ? (size_t)(n * m) * es : 0, bb = terms ? (size_t)(m * p) * es : 0;
    const size_t bc = (size_t)(n * p) * es;
    const bool d_is_c = with_d && D == C;
    if (with_d && !d_is_c) {
      const uintptr_t d0 = reinterpret_cast<uintptr_t>(D), c0 = reinterpret_cast<uintptr_t>(C);
      if (d0 < c0 + bc && c0 < d0 + bc) return MM_EINVAL;
    }
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t ob = up(ba), oc = ob + up(bb), od = oc + up(bc);
    const size_t need = od + ((with_d && !d_is_c && !dev_d) ? bc : 0);
    cudaError_t e = g_ctx.stage_ws.reserve(need, s);
    if (e != cudaSuccess) return note_cuda(e);
    uint8_t *base = static_cast<uint8_t *>(g_ctx.stage_ws.ptr);
    const void *dA = dev_a ? A : base;
    const void *dB = dev_b ? B : base + ob;
    void *dC = dev_c ? C : base + oc;
    const void *dD = !with_d ? nullptr : d_is_c ? dC : dev_d ? D : base + od;
    if (!dev_a && ba) e = cudaMemcpyAsync(base, A, ba, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !dev_b && bb) e = cudaMemcpyAsync(base + ob, B, bb, cudaMemcpyHostToDevice, s);
    // C's entries are D's where D is C: bring them in
    if (e == cudaSuccess && d_is_c && !dev_c) e = cudaMemcpyAsync(dC, C, bc, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && with_d && !d_is_c && !dev_d)
      e = cudaMemcpyAsync(base + od, D, bc, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return note_cuda(e);
    st = enqueue_axpby(n, m, p, alpha, dA, dB, beta, dD, dC, dt, mode, s);
    if (st != MM_OK) return st;
    if (!dev_c && (e = cudaMemcpyAsync(C, dC, bc, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return note_cuda(e);
    return check_device_flag(s);
  }
  st = enqueue_axpby(n, m, p, alpha, A, B, beta, D, C, dt, mode, s);
  return st != MM_OK ? st : check_device_flag(s);
}

mm_status mm_gemm(int64_t n, int64_t m, int64_t p, const void *A, const void *B, void *C,
                  mm_dtype dt, mm_mode mode) {
  MM_REQUIRE_INIT();
  mm_status st = validate(n, m, p, dt, mode);
  if (st != MM_OK) return st;
  if (n == 0 || p == 0) return MM_OK;
  if (!C || (m > 0 && (!A || !B))) return MM_EINVAL;
  std::lock_guard<std::mutex> lk(g_api_mutex);
  cudaStream_t s = g_ctx.stream;
  const size_t es = dt == MM_F64 ? 8 : 4;
  const bool dev_c = pointer_kind(C) == 1;
  const bool dev_a = m == 0 || pointer_kind(A) == 1;
  const bool dev_b = m == 0 || pointer_kind(B) == 1;
  if (dev_a && dev_b && dev_c) {
    st = enqueue_gemm(n, m, p, A, B, C, dt, mode, s);
    if (st != MM_OK) return st;
    return check_device_flag(s);
  }
  // Host operands: stage through library buffers (copies on the library
  // streams, then the same device path).
  const size_t ba = (size_t)(n * m) * es, bb = (size_t)(m * p) * es, bc = (size_t)(n * p) * es;
  const size_t oa = 0, ob = (ba + 255) & ~(size_t)255, oc = (ob + bb + 255) & ~(size_t)255;
  cudaError_t e = g_ctx.stage_ws.reserve(oc + bc, s);
  if (e != cudaSuccess) return note_cuda(e);
  uint8_t *base = static_cast<uint8_t *>(g_ctx.stage_ws.ptr);
  const void *dA = dev_a ? A : base + oa;
  const void *dB = dev_b ? B : base + ob;
  void *dC = dev_c ? C : base + oc;
  if (resolve_mode(dt, mode) == MM_MODE_SPLIT_BF16X3 && m > 0 && n >= 2048) {
    // Pipelined: B first, then slabs of A rows on the copy stream; each slab
    // is prepared and multiplied as soon as it lands (B packed once), and its
    // rows of C go back on a second copy stream while the next slab runs.
    const int chunks = (int)std::min<int64_t>(Ctx::kMaxChunks, n / 1024);
    const int64_t rc = ceil_div(ceil_div(n, chunks), kTcBM) * kTcBM;
    int64_t row0[Ctx::kMaxChunks + 1];
    for (int c = 0; c <= chunks; c++) row0[c] = std::min<int64_t>(n, c * rc);
    if (!dev_b) e = cudaMemcpyAsync(base + ob, B, bb, cudaMemcpyHostToDevice, g_ctx.h2d);
    if (e == cudaSuccess) e = cudaEventRecord(g_ctx.ev_in[0], g_ctx.h2d);
    for (int c = 0; c < chunks && e == cudaSuccess; c++) {
      const size_t off = (size_t)(row0[c] * m) * es, len = (size_t)((row0[c + 1] - row0[c]) * m) * es;
      if (!dev_a && len) e = cudaMemcpyAsync(base + oa + off, static_cast<const uint8_t *>(A) + off,
                                             len, cudaMemcpyHostToDevice, g_ctx.h2d);
      if (e == cudaSuccess) e = cudaEventRecord(g_ctx.ev_in[c + 1], g_ctx.h2d);
    }
    if (e != cudaSuccess) return note_cuda(e);
    st = run_split_chunked(g_ctx.split_ws, n, m, p, static_cast<const float *>(dA),
                           static_cast<const float *>(dB), static_cast<float *>(dC), chunks, row0, s,
                           g_ctx.ev_in, g_ctx.ev_out);
    if (st != MM_OK) return st;
    for (int c = 0; c < chunks && !dev_c && e == cudaSuccess; c++) {
      const size_t off = (size_t)(row0[c] * p) * es, len = (size_t)((row0[c + 1] - row0[c]) * p) * es;
      e = cudaStreamWaitEvent(g_ctx.d2h, g_ctx.ev_out[c], 0);
      if (e == cudaSuccess && len)
        e = cudaMemcpyAsync(static_cast<uint8_t *>(C) + off, base + oc + off, len,
                            cudaMemcpyDeviceToHost, g_ctx.d2h);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(g_ctx.d2h);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g_ctx.h2d);
    if (e != cudaSuccess) return note_cuda(e);
    return check_device_flag(s);
  }
  if (!dev_a && ba) {
    e = cudaMemcpyAsync(base + oa, A, ba, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return note_cuda(e);
  }
  if (!dev_b && bb) {
    e = cudaMemcpyAsync(base + ob, B, bb, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return note_cuda(e);
  }
  st = enqueue_gemm(n, m, p, dA, dB, dC, dt, mode, s);
  if (st != MM_OK) return st;
  if (!dev_c) {
    e = cudaMemcpyAsync(C, dC, bc, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return note_cuda(e);
  }
  return check_device_flag(s);
}

mm_status mm_gemm_grouped_async(int32_t count, const mm_problem *probs, mm_dtype dt,
                                mm_mode mode, void *stream) {
  MM_REQUIRE_INIT();
  if (count < 0 || (count > 0 && !probs)) return MM_EINVAL;
  for (int32_t g = 0; g < count; g++) {
    const mm_problem &q = probs[g];
    mm_status st = validate(q.n, q.m, q.p, dt, mode);
    if (st != MM_OK) return st;
    if (q.n == 0 || q.p == 0) continue;
    if (!q.C || (q.m > 0 && (!q.A || !q.B))) return MM_EINVAL;
  }
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : g_ctx.stream;
  std::lock_guard<std::mutex> lk(g_api_mutex);
  return enqueue_grouped(g_ctx.split_ws, g_ctx.grouped_ws, count, probs, dt,
                         resolve_mode(dt, mode), s);
}

mm_status mm_gemm_grouped(int32_t count, const mm_problem *probs, mm_dtype dt, mm_mode mode) {
  mm_status st = mm_gemm_grouped_async(count, probs, dt, mode, nullptr);
  if (st != MM_OK) return st;
  std::lock_guard<std::mutex> lk(g_api_mutex);
  return check_device_flag(g_ctx.stream);
}

mm_status mm_sync(void *stream) {
  MM_REQUIRE_INIT();
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : g_ctx.stream;
  return check_device_flag(s);
}

mm_status mm_check(int64_t n, int64_t m, int64_t p, const void *A, const void *B, const void *C,
                   mm_dtype dt, const double *x, int64_t nsamples, const int64_t *I,
                   const int64_t *J, double *out) {
  MM_REQUIRE_INIT();
  if (n < 0 || m < 0 || p < 0 || nsamples < 0 || !out) return MM_EINVAL;
  if (dt != MM_F32 && dt != MM_F64) return MM_EINVAL;
  if (n == 0 || p == 0) {
    out[0] = out[1] = 0.0;
    return MM_OK;
  }
  if (!C || !x || (m > 0 && (!A || !B)) || (nsamples > 0 && (!I || !J))) return MM_EINVAL;
  if (pointer_kind(C) != 1 || pointer_kind(x) != 1) return MM_EINVAL;
  if (m > 0 && (pointer_kind(A) != 1 || pointer_kind(B) != 1)) return MM_EINVAL;
  if (nsamples > 0 && (pointer_kind(I) != 1 || pointer_kind(J) != 1)) return MM_EINVAL;
  std::lock_guard<std::mutex> lk(g_api_mutex);
  cudaStream_t s = g_ctx.stream;
  const size_t work = check_work_doubles(n, m, p);
  cudaError_t e = g_ctx.check_ws.reserve((work + 2) * sizeof(double), s);
  if (e != cudaSuccess) return note_cuda(e);
  double *d = static_cast<double *>(g_ctx.check_ws.ptr);
  e = launch_check(dt == MM_F64, n, m, p, A, B, C, x, nsamples, I, J, d + 2, d, s);
  if (e != cudaSuccess) return note_cuda(e);
  e = cudaMemcpyAsync(out, d, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return note_cuda(e);
  e = cudaStreamSynchronize(s);
  return note_cuda(e);
}

mm_status mm_trace_enable(int on) {
  std::lock_guard<std::mutex> lk(g_trace_mu);
  g_trace_on = on != 0;
  return MM_OK;
}

mm_status mm_trace_reset(void) {
  trace_clear();
  return MM_OK;
}

mm_status mm_trace_read(const char *kernel, int64_t *launches, double *total_ms) {
  if (!kernel) return MM_EINVAL;
  std::lock_guard<std::mutex> lk(g_trace_mu);
  int64_t cnt = 0;
  double ms = 0.0;
  for (auto &r : g_trace_done) {
    if (std::strcmp(r.name, kernel) != 0) continue;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e != cudaSuccess) return from_cuda(e);
    float t = 0.f;
    e = cudaEventElapsedTime(&t, r.a, r.b);
    if (e != cudaSuccess) return from_cuda(e);
    cnt++;
    ms += t;
  }
  if (launches) *launches = cnt;
  if (total_ms) *total_ms = ms;
  return MM_OK;
}

int64_t mm_launch_count(void) { return g_launches.load(); }

}  // extern "C"
