// Library context and host-side helpers shared by api.cu, grouped.cu,
// tune.cu, serve.cu, fp8_blk.cu, tc_fused.cu, ozaki.cu and noalloc.cu.
#pragma once

#include "mm_internal.h"

namespace mm {

// Pinned host staging for problem tables: an asynchronous copy from pinned
// memory does not synchronise the host with the stream (a copy from pageable
// memory may).  The event guards reuse until the previous copy has run.
struct HostStage {
  static constexpr int kSlots = 4;  // calls the host may run ahead of the copies
  void *ptr[kSlots] = {};
  size_t bytes[kSlots] = {};
  cudaEvent_t ev[kSlots] = {};
  bool pending[kSlots] = {};
  int next = 0;
  // Copies `n` bytes from `src` to `dst` on `s` through the staging buffer.
  cudaError_t copy_to_device(void *dst, const void *src, size_t n, cudaStream_t s);
  void release();
};

// Grow-only device buffer owned by the library.
struct Scratch {
  void *ptr = nullptr;
  size_t bytes = 0;
  HostStage stage;  // host side of the tables written into this scratch
  // Makes room for `need` bytes; an existing buffer is freed after `s` has
  // drained (its contents are not kept).
  cudaError_t reserve(size_t need, cudaStream_t s);
  void release();
};

// Tile choice of the split path for one size bucket.
struct TcChoice {
  int bn;       // 128 or 256
  int bk;       // 32 or 64
  int stages;   // pipeline depth for that bk
  int group_m;  // raster band height in row tiles
  int grid;     // persistent CTAs (0 = one per SM)
  int tail = 1; // 1: split the last wave's tiles along K where the plan gains
};

// FP64 emulation (MM_MODE_OZAKI): 4-bit digit slices per operand.
constexpr int kOzakiMinSlices = 2, kOzakiMaxSlices = 12, kOzakiDefaultSlices = 12;

struct Ctx {
  bool inited = false;
  bool sticky = false;
  int device = 0;
  int sms = 0;
  mm_opts opts{};
  cudaStream_t stream = nullptr;
  int *d_err = nullptr;  // device-side timeout flag
  Scratch split_ws;      // packs, scales, tables of the split path
  Scratch fp8_ws;        // operands of the FP8 path
  Scratch grouped_ws;    // tables of the grouped SIMT path
  Scratch stage_ws;      // device copies of host operands
  Scratch check_ws;      // FP64 check work vectors
  Scratch cplx_ws;       // real/imaginary planes and partial products (mm_cgemm)
  Scratch ozaki_ws;      // digit packs, level sums and tables of the FP64 emulation
  Scratch fused_ws;      // counters and cluster partial tiles of the fused split-K path
  Scratch simt_ws;       // K-slice partials of under-filled SIMT / FP64 products
  Scratch epi_ws;        // the product of an in-place epilogue run as a second pass
  void *fused_zero_ptr = nullptr;  // fused_ws buffer whose leading counters are zero
  size_t fused_zeroed = 0;         //   and how many bytes of them
  int ozaki_slices = kOzakiDefaultSlices;  // digit slices S of MM_MODE_OZAKI
  int ozaki_gate = 1;                      // accuracy gate of MM_MODE_OZAKI on
  // host-operand pipeline of mm_gemm: copy streams and per-chunk events
  cudaStream_t h2d = nullptr, d2h = nullptr;
  cudaStream_t tc_streams[2] = {};  // slab GEMMs alternate between these
  static constexpr int kMaxChunks = 8;
  cudaEvent_t ev_in[kMaxChunks + 1] = {};
  cudaEvent_t ev_prep[kMaxChunks] = {};
  cudaEvent_t ev_out[kMaxChunks] = {};
};

extern Ctx g_ctx;
extern std::mutex g_api_mutex;

int pointer_kind(const void *p);
mm_status validate(int64_t n, int64_t m, int64_t p, mm_dtype dt, mm_mode mode);
// Queues C = A.B, or with `epi` C = alpha (A.B) + beta D (device pointers).
mm_status enqueue_gemm(int64_t n, int64_t m, int64_t p, const void *A, const void *B, void *C,
                       mm_dtype dt, mm_mode mode, cudaStream_t s, const Epi *epi = nullptr);
// Queues C = beta D for `count` entries (beta == 0: C = 0 without reading D);
// D may be C.  The epilogue of a product with no terms (alpha = 0 or m = 0).
mm_status enqueue_scale(int64_t count, double beta, const void *D, void *C, mm_dtype dt,
                        cudaStream_t s);
// Queues C = alpha A + beta B for n x p matrices (mm_add's kernels; C may be
// A or B).
mm_status enqueue_add(int64_t n, int64_t p, double alpha, const void *A, double beta,
                      const void *B, void *C, mm_dtype dt, cudaStream_t s);
mm_status check_device_flag(cudaStream_t s);

mm_status note_cuda(cudaError_t e);

// Kind of split used for inner dimension m: two bf16 parts (three products)
// where their worst-case per-product error 3 * 2^-16 is within the stated
// tolerance 1e-6 sqrt(m), three parts (six products) below that.
TcKind split_kind_for(int64_t m);
// The kind a split-path mode runs with for inner dimension m.
inline TcKind split_kind_of(mm_mode mode, int64_t m) {
  return mode == MM_MODE_SPLIT_BF16X6 ? kTcSplitBf16x6 : split_kind_for(m);
}

// N tile used for a kind: the tensor-core kernel loads B in 128-row boxes, so
// parts * bn must be a multiple of 128; with one or three parts that rules
// out bn = 64, which then becomes 128.  The three-part kind (small inner
// dimensions only) always takes bn = 128: its 128-wide layout keeps a
// four-stage ring beside the epilogue's staging buffers.
inline int tc_bn(TcKind kind, int bn) {
  if (kind == kTcSplitBf16x6) return 128;
  return (bn == 64 && pack_parts(kind) != 2) ? 128 : bn;
}

// Split path over a table of problems (single GEMM = table of one); each
// problem takes the kind split_kind_for(m).  `force` overrides the tuned tile
// choice (autotuner and tests).
// `six` selects the three-part kind (six products) for every problem.
// `epi` (null: C = A.B) is the epilogue of a table of one product.
mm_status run_split(Scratch &ws, const mm_problem *probs, int count, cudaStream_t s,
                    const TcChoice *force, bool six = false, const Epi *epi = nullptr);
// Split path for one product whose rows of A (and of C) are processed in
// `chunks` slabs: slab c waits for event in_ready[c + 1] (B: in_ready[0])
// before its prep and records out_ready[c] when its part of C is written.
// B is scaled and packed once, with slab 0.
mm_status run_split_chunked(Scratch &ws, int64_t n, int64_t m, int64_t p, const float *A,
                            const float *B, float *C, int chunks, const int64_t *row0,
                            cudaStream_t s, cudaEvent_t *in_ready, cudaEvent_t *out_ready);
// Tail split one product gets from its own shape (see tc_tail_plan), and the
// scratch bytes of its partial tiles and counters.
TcTail product_tail(int64_t n, int64_t m, int64_t p, TcKind kind, int64_t *tiles_out);
size_t tail_scratch_bytes(int64_t n, int64_t m, int64_t p, TcKind kind);
// Fused split-K path (tc_fused.cu) for products with fewer 128 x 128 tiles
// than half the SMs: S slices per tile in Q clusters of cs CTAs; S = 0 when
// the product takes the packed path.  The plan depends on the product's shape
// (and the device's cluster capacity) only.
struct FusedPlan {
  int S, Q, cs;
};
FusedPlan fused_plan(int64_t n, int64_t m, int64_t p, TcKind kind);
mm_status run_fused(Scratch &ws, int64_t n, int64_t m, int64_t p, const float *A, const float *B,
                    float *C, TcKind kind, const FusedPlan &plan, cudaStream_t s,
                    const Epi *epi = nullptr);
// FP8 path (report-only accuracy): e4m3 operands with a power-of-two scale
// per 128-value K block of each row of A and column of B (fp8_blk.cu).
mm_status run_fp8(Scratch &ws, const mm_problem *probs, int count, cudaStream_t s);
mm_status run_fp8_blocks(Scratch &ws, const mm_problem *probs, int count, cudaStream_t s);
size_t fp8_blocks_scratch_bytes(int64_t n, int64_t m, int64_t p);
// FP64 product by the Ozaki scheme on the e4m3 tensor cores with S digit
// slices (ozaki.cu); ozaki_chunk(S) = the K columns per chunk that keep every
// level sum exact in FP32; ozaki_scratch_bytes = an upper bound of the
// scratch one product needs.
// gate: check every entry against the method's error bound and recompute C
// with the FP64 FMA product where any entry could miss 1e-14 sqrt(m).
// epi (null: C = A.B) is applied by the kernels that write C.
mm_status run_ozaki(Scratch &ws, int64_t n, int64_t m, int64_t p, const double *A,
                    const double *B, double *C, int S, bool gate, cudaStream_t s,
                    const Epi *epi = nullptr);
int64_t ozaki_chunk(int S);
size_t ozaki_scratch_bytes(int64_t n, int64_t m, int64_t p, int S);
// Grouped dispatch: split / SIMT / DGEMM tables in one launch per path.
mm_status enqueue_grouped(Scratch &split_ws, Scratch &tab_ws, int count, const mm_problem *probs,
                          mm_dtype dt, mm_mode mode, cudaStream_t s);

// Autotuner table.
void tune_reset_defaults();
TcChoice tune_choose(int64_t n, int64_t m, int64_t p);
mm_status tune_load_file(const char *path);

// Serving loop.
mm_status serve_start();
void serve_stop();

}  // namespace mm
