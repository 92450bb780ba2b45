// Serving loop: continuous batching of independent products.
//
// Requests (mm_submit) queue in arrival order.  A scheduler thread admits
// them in that order while the bytes they hold on the device (operands,
// output and the library scratch they need), together with what the streams'
// buffers keep beyond the batches they run, fit the HBM budget (buffers of
// idle streams are released when the next request fits only without them),
// groups the
// admitted-but-unlaunched ones by path (split FP32, DGEMM FP64, SIMT, FP8)
// into grouped launches of at most max_batch requests and about kBatchMs of
// estimated device time (every request of a batch completes when the batch
// does, so a batch of long FP64 products would hold all of them back), and
// puts each batch on the first free stream of a small pool, so batches that
// arrive while others run overlap on the device.  A CUDA event per batch marks completion;
// the scheduler polls the events, releases the requests' bytes and stamps
// their latency (completion seen by the host - submission).
//
// Each request is computed with the tile choice of its own size (the same as
// when it runs alone), so its result does not depend on the batch it lands
// in.  With checking on, every result is followed on its stream by the FP64
// Freivalds + sampled-entries check (check.cu) and its error is reported.
//
// Not in the paper, which runs one product at a time.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <thread>
#include <unordered_map>

#include "ctx.h"

namespace mm {
namespace {

using Clock = std::chrono::steady_clock;
constexpr int kCheckSamples = 64;
constexpr int kDefaultMaxBatch = 256;
constexpr double kBatchMs = 16.0;  // estimated device time per batch (at least one request)

struct Request {
  uint64_t id = 0;
  mm_problem pr{};
  mm_dtype dt = MM_F32;
  mm_mode mode = MM_MODE_SPLIT_BF16X3;
  int slices = 0;  // MM_MODE_OZAKI: digit slices at submission
  bool gate = true;  // MM_MODE_OZAKI: accuracy gate at submission
  size_t bytes = 0;    // operands, output and the scratch estimate below
  size_t scratch = 0;  // library scratch the request needs while it runs
  Clock::time_point t_submit;
  mm_status status = MM_EPENDING;
  double err = -1.0;
  double latency_ms = 0.0;
  bool done = false;
};

// Estimated device time of a request (ms): its flops at a rough rate of its
// path on GB300.
double request_ms(const Request &r) {
  const double flops = 2.0 * (double)r.pr.n * (double)r.pr.m * (double)r.pr.p;
  double rate = 3e14;                                  // split BF16 x3 / x6
  if (r.mode == MM_MODE_DGEMM) rate = 1.2e12;          // FP64 FMA
  else if (r.mode == MM_MODE_SIMT) rate = 4.5e13;      // FP32 FMA
  else if (r.mode == MM_MODE_FP8) rate = 1e15;
  else if (r.mode == MM_MODE_SPLIT_BF16X6) rate = 1.5e14;
  else if (r.mode == MM_MODE_OZAKI) rate = 2.5e15 / (0.5 * r.slices * (r.slices + 1));
  return flops / rate * 1e3;
}

struct Slot {
  cudaStream_t s = nullptr;
  cudaEvent_t ev = nullptr;
  Scratch split_ws, tab_ws, check_ws, x_ws, idx_ws, err_ws;
  double *h_err = nullptr;     // pinned: 2 doubles per request of the batch
  int64_t *h_idx = nullptr;    // pinned: sample positions of the batch
  size_t h_cap = 0;            // requests the pinned buffers hold
  int64_t x_len = 0;           // entries of the check vector on the device
  bool busy = false;
  std::vector<Request *> batch;
  size_t batch_scratch = 0;    // scratch estimates of the batch in flight
  // Device bytes the slot's buffers hold now (they grow to the largest batch
  // the slot has run and are kept for the next one).
  size_t held() const {
    return split_ws.bytes + tab_ws.bytes + check_ws.bytes + x_ws.bytes + idx_ws.bytes +
           err_ws.bytes;
  }
  void release_buffers() {
    cudaStreamSynchronize(s);
    split_ws.release();
    tab_ws.release();
    check_ws.release();
    x_ws.release();
    idx_ws.release();
    err_ws.release();
    x_len = 0;
  }
};

struct Server {
  ~Server();
  std::thread th;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool running = false, stop = false;
  uint64_t next_id = 1;
  std::deque<Request *> pending, admitted;
  std::unordered_map<uint64_t, Request *> all;
  size_t resident = 0, budget = 0;
  int64_t completed = 0, batches = 0;
  int max_batch = kDefaultMaxBatch;
  bool check = false;
  std::vector<Slot> slots;
};

Server g_srv;

// At process exit without mm_shutdown: the scheduler may still wait on the
// condition variables that are about to be destroyed.  Stop it first; it
// leaves as soon as nothing it launched is still in flight.
Server::~Server() {
  if (!th.joinable()) return;
  {
    std::lock_guard<std::mutex> lk(mu);
    stop = true;
    pending.clear();
    admitted.clear();
  }
  cv_work.notify_all();
  th.join();
}

// SplitMix64 (Steele, Lea, Flood 2014), counter form: the check's random
// vector entries and sample positions.
uint64_t splitmix(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

size_t elem_bytes(mm_dtype dt) { return dt == MM_F64 ? 8 : 4; }

// Library scratch a request needs while it runs (split: bf16 hi/lo packs
// padded to whole tiles, scale words, tail-split partial tiles; FP64
// emulation: digit packs and level sums).
size_t request_scratch(const mm_problem &q, mm_mode mode, int slices) {
  size_t b = 0;
  if (mode == MM_MODE_OZAKI) b += ozaki_scratch_bytes(q.n, q.m, q.p, slices);
  if (mode == MM_MODE_FP8) b += fp8_blocks_scratch_bytes(q.n, q.m, q.p);
  if (mode == MM_MODE_SPLIT_BF16X3 || mode == MM_MODE_SPLIT_BF16X6) {
    const TcKind kind = split_kind_of(mode, q.m);
    TcChoice c = tune_choose(q.n, q.m, q.p);
    c.bn = tc_bn(kind, c.bn);
    const size_t kb = (size_t)ceil_div(q.m, pack_k(kind));  // pack rows per matrix row
    b += (size_t)kPackRowBytes * pack_parts(kind) * kb *
         ((size_t)ceil_div(q.n, kTcBM) * kTcBM + (size_t)ceil_div(q.p, c.bn) * c.bn);
    b += 4 * (size_t)(q.n + q.p) + sizeof(SplitProb);
    b += tail_scratch_bytes(q.n, q.m, q.p, kind);  // partial tiles of a tail split
  }
  return b;
}

// Device bytes of a request's operands and output (the caller's memory).
size_t request_operand_bytes(const mm_problem &q, mm_dtype dt) {
  return elem_bytes(dt) * (size_t)(q.n * q.m + q.m * q.p + q.n * q.p);
}

// Bytes the slots' buffers hold beyond the scratch estimates of the batches
// they run: what a slot kept from an earlier, larger batch (or an idle slot's
// buffers).  Counted against the budget with the admitted requests.
size_t slots_extra() {
  size_t x = 0;
  for (const Slot &sl : g_srv.slots) {
    const size_t h = sl.held();
    x += h > sl.batch_scratch ? h - sl.batch_scratch : 0;
  }
  return x;
}

// Whether the request at the head of the queue fits the budget now; if it
// fits only without the buffers that idle slots keep, those are released.
bool head_fits() {
  const size_t need = g_srv.pending.front()->bytes;
  if (g_srv.resident + slots_extra() + need <= g_srv.budget) return true;
  if (g_srv.resident + need > g_srv.budget) return false;
  bool freed = false;
  for (Slot &sl : g_srv.slots)
    if (!sl.busy && sl.held() > 0) {
      sl.release_buffers();
      freed = true;
    }
  return freed && g_srv.resident + slots_extra() + need <= g_srv.budget;
}

void finish(Request *r, mm_status st, double err) {
  r->status = st;
  r->err = err;
  r->latency_ms =
      std::chrono::duration<double, std::milli>(Clock::now() - r->t_submit).count();
  r->done = true;
}

// Launches one batch (requests of one path) on a slot.  Caller holds mu.
mm_status launch_batch(Slot &sl, std::vector<Request *> &reqs) {
  std::vector<mm_problem> probs;
  probs.reserve(reqs.size());
  for (Request *r : reqs) probs.push_back(r->pr);
  const mm_dtype dt = reqs[0]->dt;
  const mm_mode mode = reqs[0]->mode;
  mm_status st;
  if (mode == MM_MODE_SPLIT_BF16X3 || mode == MM_MODE_SPLIT_BF16X6)
    st = run_split(sl.split_ws, probs.data(), (int)probs.size(), sl.s, nullptr,
                   mode == MM_MODE_SPLIT_BF16X6);
  else if (mode == MM_MODE_FP8)
    st = run_fp8(sl.split_ws, probs.data(), (int)probs.size(), sl.s);
  else if (mode == MM_MODE_OZAKI) {
    // one emulated product after the other on the slot's stream
    st = MM_OK;
    for (size_t k = 0; k < reqs.size() && st == MM_OK; k++) {
      const mm_problem &q = reqs[k]->pr;
      st = run_ozaki(sl.split_ws, q.n, q.m, q.p, static_cast<const double *>(q.A),
                     static_cast<const double *>(q.B), static_cast<double *>(q.C),
                     reqs[k]->slices, reqs[k]->gate, sl.s);
    }
  } else
    st = enqueue_grouped(sl.split_ws, sl.tab_ws, (int)probs.size(), probs.data(), dt, mode, sl.s);
  if (st != MM_OK) return st;
  if (g_srv.check) {
    const size_t k = reqs.size();
    if (k > sl.h_cap) {
      if (sl.h_err) cudaFreeHost(sl.h_err);
      if (sl.h_idx) cudaFreeHost(sl.h_idx);
      sl.h_err = nullptr;
      sl.h_idx = nullptr;
      sl.h_cap = 0;
      if (cudaMallocHost(&sl.h_err, 2 * k * sizeof(double)) != cudaSuccess ||
          cudaMallocHost(&sl.h_idx, 2 * k * kCheckSamples * sizeof(int64_t)) != cudaSuccess)
        return MM_ENOMEM;
      sl.h_cap = k;
    }
    int64_t maxp = 0, maxm = 1;
    for (Request *r : reqs) {
      maxp = std::max<int64_t>(maxp, r->pr.p);
      maxm = std::max<int64_t>(maxm, r->pr.m);
    }
    cudaError_t e;
    if (maxp > sl.x_len) {
      if ((e = sl.x_ws.reserve((size_t)maxp * sizeof(double), sl.s)) != cudaSuccess)
        return from_cuda(e);
      std::vector<double> x((size_t)maxp);
      for (int64_t j = 0; j < maxp; j++)
        x[(size_t)j] = (double)(int64_t)(splitmix(0x5EEDull, (uint64_t)j) >> 11) * 0x1p-52 - 1.0;
      if ((e = cudaMemcpy(sl.x_ws.ptr, x.data(), (size_t)maxp * sizeof(double),
                          cudaMemcpyHostToDevice)) != cudaSuccess)
        return from_cuda(e);
      sl.x_len = maxp;
    }
    if ((e = sl.idx_ws.reserve(2 * k * kCheckSamples * sizeof(int64_t), sl.s)) != cudaSuccess ||
        (e = sl.err_ws.reserve(2 * k * sizeof(double), sl.s)) != cudaSuccess ||
        (e = sl.check_ws.reserve(check_work_doubles(1, maxm, 1) * sizeof(double), sl.s)) !=
            cudaSuccess)
      return from_cuda(e);
    for (size_t q = 0; q < k; q++) {
      const Request *r = reqs[q];
      for (int t = 0; t < kCheckSamples; t++) {
        const uint64_t u = splitmix(r->id, (uint64_t)t);
        sl.h_idx[(2 * q) * kCheckSamples + t] = (int64_t)(u % (uint64_t)r->pr.n);
        sl.h_idx[(2 * q + 1) * kCheckSamples + t] = (int64_t)((u >> 32) % (uint64_t)r->pr.p);
      }
    }
    int64_t *d_idx = static_cast<int64_t *>(sl.idx_ws.ptr);
    double *d_err = static_cast<double *>(sl.err_ws.ptr);
    if ((e = cudaMemcpyAsync(d_idx, sl.h_idx, 2 * k * kCheckSamples * sizeof(int64_t),
                             cudaMemcpyHostToDevice, sl.s)) != cudaSuccess)
      return from_cuda(e);
    for (size_t q = 0; q < k; q++) {
      const Request *r = reqs[q];
      if (r->pr.n == 0 || r->pr.p == 0) {
        cudaMemsetAsync(d_err + 2 * q, 0, 2 * sizeof(double), sl.s);
        continue;
      }
      e = launch_check(r->dt == MM_F64, r->pr.n, r->pr.m, r->pr.p, r->pr.A, r->pr.B, r->pr.C,
                       static_cast<const double *>(sl.x_ws.ptr), kCheckSamples,
                       d_idx + (2 * q) * kCheckSamples, d_idx + (2 * q + 1) * kCheckSamples,
                       static_cast<double *>(sl.check_ws.ptr), d_err + 2 * q, sl.s);
      if (e != cudaSuccess) return from_cuda(e);
    }
    if ((e = cudaMemcpyAsync(sl.h_err, d_err, 2 * k * sizeof(double), cudaMemcpyDeviceToHost,
                             sl.s)) != cudaSuccess)
      return from_cuda(e);
  }
  cudaError_t e = cudaEventRecord(sl.ev, sl.s);
  return from_cuda(e);
}

void scheduler() {
  std::unique_lock<std::mutex> lk(g_srv.mu);
  cudaSetDevice(g_ctx.device);
  for (;;) {
    // 1. completions
    for (Slot &sl : g_srv.slots) {
      if (!sl.busy) continue;
      const cudaError_t q = cudaEventQuery(sl.ev);
      if (q == cudaErrorNotReady) continue;
      mm_status st = q == cudaSuccess ? MM_OK : MM_ECUDA;
      if (q != cudaSuccess) cudaGetLastError();
      for (size_t k = 0; k < sl.batch.size(); k++) {
        Request *r = sl.batch[k];
        double err = -1.0;
        if (g_srv.check && st == MM_OK) err = std::max(sl.h_err[2 * k], sl.h_err[2 * k + 1]);
        finish(r, st, err);
        g_srv.resident -= r->bytes;
        g_srv.completed++;
      }
      sl.batch.clear();
      sl.batch_scratch = 0;
      sl.busy = false;
      g_srv.cv_done.notify_all();
    }
    // 2. admission in arrival order while the budget allows
    while (!g_srv.pending.empty() && head_fits()) {
      Request *r = g_srv.pending.front();
      g_srv.pending.pop_front();
      g_srv.resident += r->bytes;
      g_srv.admitted.push_back(r);
    }
    // 3. batches onto free streams: the path of the oldest admitted request,
    // its requests in arrival order up to max_batch and ~kBatchMs of work
    for (Slot &sl : g_srv.slots) {
      if (sl.busy || g_srv.admitted.empty()) continue;
      const mm_mode mode = g_srv.admitted.front()->mode;
      const mm_dtype dt = g_srv.admitted.front()->dt;
      std::vector<Request *> take;
      std::deque<Request *> rest;
      double ms = 0.0;
      bool full = false;
      for (Request *r : g_srv.admitted) {
        if (!full && r->mode == mode && r->dt == dt) {
          const double c = request_ms(*r);
          if ((int)take.size() < g_srv.max_batch && (take.empty() || ms + c <= kBatchMs)) {
            take.push_back(r);
            ms += c;
            continue;
          }
          full = true;  // later requests of this path wait for the next batch
        }
        rest.push_back(r);
      }
      g_srv.admitted.swap(rest);
      const mm_status st = launch_batch(sl, take);
      if (st != MM_OK) {
        cudaGetLastError();
        for (Request *r : take) {
          finish(r, st, -1.0);
          g_srv.resident -= r->bytes;
          g_srv.completed++;
        }
        g_srv.cv_done.notify_all();
        continue;
      }
      sl.batch_scratch = 0;
      for (const Request *r : take) sl.batch_scratch += r->scratch;
      sl.batch = std::move(take);
      sl.busy = true;
      g_srv.batches++;
    }
    // 4. exit once stopped and drained
    bool inflight = false;
    for (Slot &sl : g_srv.slots) inflight = inflight || sl.busy;
    if (g_srv.stop && !inflight) break;
    // 5. sleep until new work, or poll the events shortly
    if (inflight)
      g_srv.cv_work.wait_for(lk, std::chrono::microseconds(20));
    else
      g_srv.cv_work.wait(lk, [] {
        return g_srv.stop || (!g_srv.pending.empty() && head_fits()) ||
               !g_srv.admitted.empty();
      });
  }
}

}  // namespace

mm_status serve_start() {
  std::lock_guard<std::mutex> lk(g_srv.mu);
  if (g_srv.running) return MM_OK;
  g_srv.stop = false;
  for (auto &kv : g_srv.all) delete kv.second;
  g_srv.all.clear();
  g_srv.pending.clear();
  g_srv.admitted.clear();
  g_srv.budget = g_ctx.opts.hbm_budget_bytes;
  g_srv.max_batch = g_ctx.opts.max_batch > 0 ? g_ctx.opts.max_batch : kDefaultMaxBatch;
  g_srv.check = g_ctx.opts.check != 0;
  g_srv.resident = 0;
  g_srv.completed = 0;
  g_srv.batches = 0;
  g_srv.slots.clear();
  g_srv.slots.resize((size_t)g_ctx.opts.n_streams);
  for (Slot &sl : g_srv.slots) {
    if (cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess)
      return MM_ECUDA;
  }
  g_srv.running = true;
  g_srv.th = std::thread(scheduler);
  return MM_OK;
}

void serve_stop() {
  {
    std::lock_guard<std::mutex> lk(g_srv.mu);
    if (!g_srv.running) return;
    g_srv.stop = true;
    // requests not yet launched are cancelled
    for (auto *q : {&g_srv.pending, &g_srv.admitted}) {
      for (Request *r : *q) {
        if (q == &g_srv.admitted) g_srv.resident -= r->bytes;
        finish(r, MM_ECANCELLED, -1.0);
      }
      q->clear();
    }
    g_srv.cv_work.notify_all();
  }
  g_srv.th.join();
  std::lock_guard<std::mutex> lk(g_srv.mu);
  for (Slot &sl : g_srv.slots) {
    sl.release_buffers();
    if (sl.h_err) cudaFreeHost(sl.h_err);
    if (sl.h_idx) cudaFreeHost(sl.h_idx);
    cudaEventDestroy(sl.ev);
    cudaStreamDestroy(sl.s);
  }
  g_srv.slots.clear();
  // finished requests stay pollable until the next start
  g_srv.running = false;
  g_srv.cv_done.notify_all();
}

}  // namespace mm

using namespace mm;

extern "C" {

mm_status mm_submit(const mm_problem *pr, mm_dtype dt, mm_mode mode, uint64_t *id_out) {
  if (!g_ctx.inited) return MM_ENOTINIT;
  if (g_ctx.sticky) return MM_ECUDA;
  if (!pr || !id_out) return MM_EINVAL;
  mm_status st = validate(pr->n, pr->m, pr->p, dt, mode);
  if (st != MM_OK) return st;
  if (mode == MM_MODE_AUTO) mode = dt == MM_F64 ? MM_MODE_DGEMM : MM_MODE_SPLIT_BF16X3;
  if (pr->n > 0 && pr->p > 0) {
    if (!pr->C || pointer_kind(pr->C) != 1) return MM_EINVAL;
    if (pr->m > 0 && (!pr->A || !pr->B || pointer_kind(pr->A) != 1 || pointer_kind(pr->B) != 1))
      return MM_EINVAL;
  }
  Request *r = new Request();
  r->pr = *pr;
  r->dt = dt;
  r->mode = mode;
  r->slices = g_ctx.ozaki_slices;
  r->gate = g_ctx.ozaki_gate != 0;
  r->scratch = request_scratch(*pr, mode, r->slices);
  r->bytes = request_operand_bytes(*pr, dt) + r->scratch;
  std::lock_guard<std::mutex> lk(g_srv.mu);
  if (!g_srv.running) {
    delete r;
    return MM_ENOTINIT;
  }
  if (r->bytes > g_srv.budget) {
    delete r;
    return MM_EBUDGET;
  }
  r->id = g_srv.next_id++;
  r->t_submit = Clock::now();
  g_srv.all[r->id] = r;
  g_srv.pending.push_back(r);
  g_srv.cv_work.notify_one();
  *id_out = r->id;
  return MM_OK;
}

static mm_status take_result(uint64_t id, mm_status *result, double *err, double *lat) {
  auto it = g_srv.all.find(id);
  if (it == g_srv.all.end()) return MM_ENOTFOUND;
  Request *r = it->second;
  if (!r->done) return MM_EPENDING;
  if (result) *result = r->status;
  if (err) *err = r->err;
  if (lat) *lat = r->latency_ms;
  g_srv.all.erase(it);
  delete r;
  return MM_OK;
}

mm_status mm_poll(uint64_t id, mm_status *result, double *err_out, double *latency_ms_out) {
  std::lock_guard<std::mutex> lk(g_srv.mu);
  return take_result(id, result, err_out, latency_ms_out);
}

mm_status mm_wait(uint64_t id, double timeout_s, mm_status *result, double *err_out,
                  double *latency_ms_out) {
  std::unique_lock<std::mutex> lk(g_srv.mu);
  const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                        std::chrono::duration<double>(timeout_s));
  for (;;) {
    auto it = g_srv.all.find(id);
    if (it == g_srv.all.end()) return MM_ENOTFOUND;
    if (it->second->done) return take_result(id, result, err_out, latency_ms_out);
    if (g_srv.cv_done.wait_until(lk, until) == std::cv_status::timeout) {
      auto it2 = g_srv.all.find(id);
      if (it2 != g_srv.all.end() && it2->second->done)
        return take_result(id, result, err_out, latency_ms_out);
      return MM_ETIMEOUT;
    }
  }
}

mm_status mm_serve_stats(int64_t *completed, int64_t *batches, int64_t *waiting,
                         int64_t *resident_bytes) {
  std::lock_guard<std::mutex> lk(g_srv.mu);
  if (completed) *completed = g_srv.completed;
  if (batches) *batches = g_srv.batches;
  if (waiting) *waiting = (int64_t)(g_srv.pending.size() + g_srv.admitted.size());
  if (resident_bytes) *resident_bytes = (int64_t)(g_srv.resident + slots_extra());
  return MM_OK;
}

}  // extern "C"
