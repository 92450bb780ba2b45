/*
 * mm.h - C ABI of the GB300 dense matrix-product library.
 *
 * The library computes the Cauchy product C = A.B of a row-major n x m matrix
 * A and a row-major m x p matrix B:
 *
 *     c_ij = sum_{r=1..m} a_ir * b_rj,   1 <= i <= n, 1 <= j <= p
 *
 * (paper: Swierczewski, "Akceleracja obliczen algebry liniowej ...", Section
 * "Implementacje algorytmow", the definition of the Cauchy product; storage
 * as in its Listing 1: A[i*m + k], B[k*p + j], C[i*p + j]).  All matrices are
 * dense: the leading dimension is the number of columns.
 *
 * Paths (selected by mm_mode):
 *   MM_MODE_SIMT          FP32 in/out, FP32 FMA on the CUDA cores, shared-
 *                         memory tiled with register blocking.  The paper's
 *                         Listing 4 (shared-memory tiling) is its ancestor.
 *                         Each entry is summed in ascending r by one thread;
 *                         a product with too few output tiles for the SMs
 *                         (from its shape alone) is cut along K into slices
 *                         whose partial sums are then added in a fixed order.
 *   MM_MODE_SPLIT_BF16X3  FP32 in/out on the tensor cores: every operand is
 *                         scaled per row (A) / per column (B) by a power of
 *                         two and split into bf16 hi + lo parts; the product
 *                         is accumulated in FP32 as hi.hi + hi.lo + lo.hi
 *                         (tcgen05 MMA, accumulator in tensor memory) and
 *                         unscaled exactly.  Not in the paper.
 *   MM_MODE_DGEMM         FP64 in/out, FP64 FMA (K slices as for
 *                         MM_MODE_SIMT).  The paper's Table 2 "double" column
 *                         computes this product in double.
 *   MM_MODE_FP8           FP32 in/out through e4m3 operands: each row of A
 *                         and column of B is cut into K blocks of 128 values,
 *                         each block scaled by its own power of two (largest
 *                         magnitude to [128, 256)); every block's product is
 *                         accumulated on the tensor cores, unscaled exactly
 *                         and added in FP32.  Accuracy is reported, not
 *                         guaranteed.  Not in the paper.
 *   MM_MODE_SPLIT_BF16X6  FP32 in/out on the tensor cores, the upper rung
 *                         of the split ladder: three bf16 parts (hi, mid,
 *                         lo) per scaled operand and the six products down to
 *                         2^-16 relative (mid.mid, hi.lo, lo.hi, hi.mid,
 *                         mid.hi, hi.hi), so every term keeps about FP32
 *                         precision; about half the rate of SPLIT_BF16X3.
 *                         SPLIT_BF16X3 itself takes this form for inner
 *                         dimensions m < 2237, where two parts cannot meet its
 *                         tolerance.  Not in the paper.
 *   MM_MODE_AUTO          SPLIT_BF16X3 for MM_F32, DGEMM for MM_F64.
 *   MM_MODE_OZAKI         FP64 in/out on the e4m3 tensor cores (Ozaki
 *                         scheme): each row of A / column of B is scaled by a
 *                         power of two and cut into S balanced base-32
 *                         integer digit slices (|d| <= 16); the slice
 *                         products of equal weight are
 *                         exact in FP32; the levels are added exactly in
 *                         128-bit integers and rounded once to FP64.  Accuracy
 *                         depends on S and on the spread of magnitudes within
 *                         rows and columns (mm_ozaki_slices).  Not in the
 *                         paper.
 *
 * Accuracy contract (measured against an FP64 CPU evaluation of the
 * definition): max_ij |c^_ij - c_ij| / (|A|.|B|)_ij <= 1e-6*sqrt(m) for SIMT
 * SPLIT_BF16X3 and SPLIT_BF16X6, <= 1e-14*sqrt(m) for DGEMM, for finite inputs whose
 * products stay in range.
 *
 * Conventions for every entry point:
 *   - Return value: MM_OK or an error code; no function aborts or prints.
 *   - Device pointers are CUDA device (or managed) memory of the library's
 *     device.  mm_gemm also accepts host pointers (pageable or pinned): it
 *     then stages the operands through library-owned device buffers.
 *   - The caller owns A, B, C.  The library owns its scratch: packed bf16
 *     operand splits, scale exponents, problem tables, tensor memory.
 *   - n, m, p >= 0.  n == 0 or p == 0 is a no-op; m == 0 writes C = 0.
 *   - dtype/mode mismatch (MM_F64 with SIMT/SPLIT_BF16X3/SPLIT_BF16X6/FP8,
 *     MM_F32 with DGEMM or OZAKI) returns MM_EUNSUPPORTED.
 *   - A sticky CUDA error (the context is lost) returns MM_ECUDA from then on.
 *   - Device-side waits are bounded; a wait that runs out sets a device flag
 *     that the next synchronising call reports as MM_ETIMEOUT.
 *   - Not thread-safe except mm_submit / mm_poll / mm_wait, which may be
 *     called from any thread while the serving loop runs.
 */
#ifndef MM_H
#define MM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MM_OK = 0,
  MM_EINVAL = 1,       /* bad argument (negative size, null pointer, ...) */
  MM_ENOMEM = 2,       /* device or host allocation failed */
  MM_EBUDGET = 3,      /* request larger than the serving HBM budget */
  MM_EBUSY = 4,        /* mm_init called twice */
  MM_ENOTFOUND = 5,    /* unknown request id */
  MM_EPENDING = 6,     /* request not finished yet */
  MM_ETIMEOUT = 7,     /* a bounded wait ran out (device or host side) */
  MM_ECUDA = 8,        /* CUDA runtime/driver error */
  MM_ENOTINIT = 9,     /* mm_init not called */
  MM_EUNSUPPORTED = 10,/* dtype/mode combination or device not supported */
  MM_ECANCELLED = 11,  /* request cancelled by mm_shutdown */
  MM_ESCRATCH = 12     /* product too large for mm_gemm_split_static's fixed
                          scratch array */
} mm_status;

typedef enum { MM_F32 = 0, MM_F64 = 1 } mm_dtype;

typedef enum {
  MM_MODE_SIMT = 0,
  MM_MODE_SPLIT_BF16X3 = 1,
  MM_MODE_DGEMM = 2,
  MM_MODE_FP8 = 3,
  MM_MODE_AUTO = 4,
  MM_MODE_OZAKI = 5,
  MM_MODE_SPLIT_BF16X6 = 6
} mm_mode;

typedef struct {
  size_t hbm_budget_bytes; /* serving admission budget; 0 selects 40 GiB */
  int n_streams;           /* serving streams; 0 selects 2 */
  const char *tune_table;  /* autotuner table to load; NULL: built-in choice */
  int check;               /* 1: the serving loop checks every result on the
                              GPU (Freivalds + sampled entries, FP64) */
  int device;              /* CUDA device ordinal; -1 keeps the current one */
  int max_batch;           /* serving: most requests per grouped launch; 0
                              selects 256, 1 gives one request per launch */
} mm_opts;

/* One independent product C = A.B (row-major, dense; see conventions). */
typedef struct {
  int64_t n, m, p;
  const void *A;
  const void *B;
  void *C;
} mm_problem;

/* Library set-up.  opts may be NULL (defaults).  Selects the device, creates
 * the library stream and checks that the device is sm_103 (B300 class).
 * Returns MM_EBUSY if already initialised, MM_EUNSUPPORTED on another GPU. */
mm_status mm_init(const mm_opts *opts);

/* Stops the serving loop: requests not yet launched end MM_ECANCELLED,
 * launched ones finish; their final status stays pollable until the next
 * mm_init.  Waits for the library's streams and frees every library
 * allocation.  Idempotent. */
mm_status mm_shutdown(void);

/* Static string for a status code. */
const char *mm_strerror(mm_status s);

/* C = A.B (paper: definition of the Cauchy product; Listing 1 storage).
 * A: n x m, B: m x p, C: n x p of dtype dt, row-major and dense.  Device or
 * host pointers (host: staged through library buffers).  Synchronous: returns
 * when C is written.  C is fully overwritten and must not alias A or B. */
mm_status mm_gemm(int64_t n, int64_t m, int64_t p, const void *A, const void *B,
                  void *C, mm_dtype dt, mm_mode mode);

/* Digit slices S used by MM_MODE_OZAKI for products queued after the call
 * (serving requests keep the value current at mm_submit).  2 <= S <= 12,
 * default 12; the cost grows as S (S + 1) / 2 e4m3 products.
 * Method (K. Ozaki, T. Ogita, S. Oishi, S. M. Rump, Numer. Algorithms 59,
 * 2012, error-free splitting of matrix products): with sigma_i =
 * ilogb(max_r |a_ir|) + 2 and tau_j likewise for column j of B, every entry
 * is truncated to 5S bits below 2^sigma and written as S balanced base-32
 * digits (d_0 in [0, 16], the others in [-16, 15], signed by the entry;
 * exact in e4m3); level L = t + u of the digit products is one tensor-core
 * product whose FP32 sums stay exact (K is cut into chunks of at most
 * (2^24 - 1) / (256 S) columns for that); levels t + u >= S are dropped.
 * Each term a_ir b_rj is then off by at most
 * (S + 2) 2^(sigma_i + tau_j - 5S - 1), zero entries by nothing: relative to
 * (|A||B|)_ij about 8 (S + 2) 2^(-5S) (S = 12: 1e-16) for rows and columns
 * without a wide spread of magnitudes, more where a row's largest entry
 * dwarfs the entries that meet the column's mass (the accuracy gate below
 * guards the FP64 tolerance).  Rows of A or columns of B holding a NaN or an
 * infinity give NaN rows or columns of C.  Scratch: (S + 1 digit bytes per
 * entry of A and B, plus S + 1 FP32 level sums per entry of C per K chunk),
 * library-owned.  Returns MM_EINVAL outside 2..12, MM_ENOTINIT before
 * mm_init.  An MM_MODE_OZAKI product whose inner dimension needs more than
 * 1024 K chunks (m above about 5.5 million at S = 12) returns MM_EINVAL. */
mm_status mm_ozaki_slices(int slices);

/* Accuracy gate of MM_MODE_OZAKI products queued after the call (serving
 * requests keep the setting current at mm_submit); on (1) by default.  Entry
 * (i, j) of the emulation is off by at most
 * m (S + 2) 2^(sigma_i + tau_j - 5S - 1)
 * (scales 2^sigma_i of row i of A, 2^tau_j of column j of B), so it meets
 * 1e-14 sqrt(m) of (|A||B|)_ij wherever P_ij = sum_r |a_ir| 2^-sigma_i
 * |b_rj| 2^-tau_j >= sqrt(m) (S + 2) 2^(-5S-1) 1e14.  With the gate, each product
 * also packs one more e4m3 slice per operand (16 |x| 2^-sigma truncated
 * toward zero onto the e4m3 grid) and multiplies the two on the tensor cores,
 * a lower bound of 256 P, and checks every entry against the threshold
 * divided by 0.98 - m 2^-23 (room for the FP32 accumulation and the final
 * rounding; every product falls back where m 2^-23 > 0.48).  If any entry
 * with a finite, non-zero row and column misses it (magnitudes spread over
 * many binades, entries below the e4m3 grid), the FP64 FMA product
 * (MM_MODE_DGEMM's kernel) recomputes all of C on the device, so the result
 * meets the FP64 tolerance for any finite input; the decision is
 * data-dependent and made on the device (no host round trip).  Off (0): the
 * emulation's result is returned as it is (bit for bit the method of
 * mm_ozaki_slices; the gate never changes the emulation's own bits).
 * Returns MM_EINVAL for other values, MM_ENOTINIT before mm_init. */
mm_status mm_ozaki_gate(int on);

/* Plan of an MM_MODE_OZAKI product, a pure host function (no device, no
 * mm_init): for A n x m, B m x p and `slices` digit slices, writes the K
 * columns per chunk (the largest multiple of 128 with
 * 256 * slices * columns < 2^24, so every level sum stays an exact FP32
 * integer), the number of chunks (ceil(m / columns); 0 for m = 0) and an
 * upper bound of the library scratch the product holds (digit packs, FP32
 * level sums, maxima, table).  Returns MM_EINVAL for negative sizes, slices
 * outside 2..12, NULL outputs or more than 1024 chunks. */
mm_status mm_ozaki_plan(int64_t n, int64_t m, int64_t p, int slices, int64_t *chunk_columns,
                        int *chunks, size_t *scratch_bytes);

/* As mm_gemm, but device pointers only and asynchronous: the work is queued on
 * `stream` (a cudaStream_t; NULL = the library stream) and the call returns
 * after the launches.  Calls that use the split, FP8 or Ozaki path share the
 * library's scratch of that path and must be ordered on one stream; so must
 * SIMT and DGEMM calls on products with too few output tiles for the SMs,
 * whose K slices keep their partial sums in library scratch. */
mm_status mm_gemm_async(int64_t n, int64_t m, int64_t p, const void *A,
                        const void *B, void *C, mm_dtype dt, mm_mode mode,
                        void *stream);

/* C = alpha (A.B) + beta D for one product: the paper's second workload, the
 * elementwise matrix addition/subtraction of the results section, fused into
 * the epilogue of the product on the SIMT, DGEMM, split and FP64-emulation
 * paths (the kernel that writes C applies it to each entry as it stores it,
 * so D is read once and no second pass over C runs; the tensor-core kernels
 * keep their tiled stores where C and D are 16-byte aligned with p % 4 == 0).
 * mm_gemm_axpby takes device or host pointers (host operands are staged
 * through library buffers, as mm_gemm does); mm_gemm_axpby_async takes device
 * pointers only.  D is n x p row-major like C, of the same dtype, and
 * is either C itself (C = alpha (A.B) + beta C) or apart from it (a partial
 * overlap returns MM_EINVAL).  Each entry x of the product (computed by
 * `mode` as mm_gemm does) becomes fma(alpha, x, beta d) with one rounding of
 * beta d first, in the element type (MM_F32: alpha and beta rounded to FP32);
 * alpha = 1 and beta = +-1 give x +- d correctly rounded, and beta = 0 gives
 * alpha x without reading D (D may be NULL).  alpha = 0 or m = 0: C = beta D,
 * and A and B are not read (they may be NULL).  With alpha = 1 and beta = 0
 * the result is mm_gemm's, bit for bit.  MM_MODE_FP8 runs the same
 * arithmetic as one elementwise pass after the product instead (its e4m3
 * tiles' MMAs take about as long as their stores, so the tensor-core kernel
 * has no slack for it); with D = C the product then goes to library scratch
 * first.  Returns
 * what mm_gemm returns, plus MM_EINVAL for a NULL D where beta != 0 (and,
 * from the asynchronous form, for a host D).
 * mm_gemm_axpby waits for the result; mm_gemm_axpby_async queues it on
 * `stream` (NULL = the library stream) under mm_gemm_async's scratch rule. */
mm_status mm_gemm_axpby(int64_t n, int64_t m, int64_t p, double alpha, const void *A,
                        const void *B, double beta, const void *D, void *C, mm_dtype dt,
                        mm_mode mode);
mm_status mm_gemm_axpby_async(int64_t n, int64_t m, int64_t p, double alpha, const void *A,
                              const void *B, double beta, const void *D, void *C,
                              mm_dtype dt, mm_mode mode, void *stream);

/* count independent products in one persistent launch per path (grouped
 * GEMM).  probs is a host array; A/B/C inside it are device pointers.  Tile
 * shapes and raster order come from the autotuner table.  Synchronous.
 * MM_MODE_OZAKI products run one after the other (each its own launches). */
mm_status mm_gemm_grouped(int32_t count, const mm_problem *probs, mm_dtype dt,
                          mm_mode mode);
mm_status mm_gemm_grouped_async(int32_t count, const mm_problem *probs,
                                mm_dtype dt, mm_mode mode, void *stream);

/* Waits for `stream` (NULL = library stream) and reports a device-side
 * timeout flag (MM_ETIMEOUT) or a CUDA error raised by earlier async calls. */
mm_status mm_sync(void *stream);

/* FP64 check of a computed product on the GPU.
 * Freivalds' test: y = C.x and z = A.(B.x) in FP64 with x (device, length p,
 * FP64) given; out[0] = max_i |y_i - z_i| / (|A|.(|B|.|x|))_i.
 * Sampled entries: for t < nsamples, (I[t], J[t]) (device int64 arrays):
 * out[1] = max_t |C_IJ - (A.B)_IJ| / (|A|.|B|)_IJ with the dot product in
 * FP64.  out (host, 2 doubles) receives both; a zero normaliser with a
 * non-zero difference gives +inf.  dt gives the element type of A, B, C.
 * Synchronous. */
mm_status mm_check(int64_t n, int64_t m, int64_t p, const void *A,
                   const void *B, const void *C, mm_dtype dt, const double *x,
                   int64_t nsamples, const int64_t *I, const int64_t *J,
                   double *out);

/* ----------------------------------------------------------------- serving */

/* Queues one request (device pointers; they must stay valid until mm_poll or
 * mm_wait reports a final status).  Admission: the request's operand, output
 * and scratch bytes, with those of the requests already admitted and the
 * buffers the serving streams keep, must fit the HBM budget (idle streams
 * give their buffers back when that makes the request fit); a request that
 * can never fit returns MM_EBUDGET immediately.  Requests are batched by dtype and mode;
 * a batch of MM_MODE_OZAKI requests runs them one after the other on its
 * stream.  *id_out receives the request id. */
mm_status mm_submit(const mm_problem *pr, mm_dtype dt, mm_mode mode,
                    uint64_t *id_out);

/* Non-blocking status of a request.  Returns MM_EPENDING while queued or
 * running, MM_ENOTFOUND for an unknown id, else MM_OK with *result = the
 * product's own status, *err_out = the GPU check's max normalised error (or
 * -1 when checking is off), *latency_ms_out = completion - submission time.
 * A request is forgotten after its final status has been returned once. */
mm_status mm_poll(uint64_t id, mm_status *result, double *err_out,
                  double *latency_ms_out);

/* Blocks until the request finishes or timeout_s passes (MM_ETIMEOUT); then
 * as mm_poll. */
mm_status mm_wait(uint64_t id, double timeout_s, mm_status *result,
                  double *err_out, double *latency_ms_out);

/* Serving counters: completed requests, batches launched, requests waiting,
 * and the device bytes counted against the HBM budget now (operands, outputs
 * and scratch of the admitted requests, plus what the serving streams'
 * buffers keep from earlier, larger batches).  Any pointer may be NULL. */
mm_status mm_serve_stats(int64_t *completed, int64_t *batches,
                         int64_t *waiting, int64_t *resident_bytes);

/* --------------------------------------------------------------- autotuner */

/* Times the candidate tile configurations of the split path for products of
 * size n x m x p on the device (scratch operands, reps repetitions each) and
 * records the fastest for the size bucket of (n, m, p).  Synchronous. */
mm_status mm_tune(int64_t n, int64_t m, int64_t p, int reps);

/* Writes / reads the tuning table (text, one bucket per line). */
mm_status mm_tune_save(const char *path);
mm_status mm_tune_load(const char *path);

/* Tile configuration the split path would use for (n, m, p): block N width,
 * K depth, pipeline stages and raster group height. */
mm_status mm_tune_query(int64_t n, int64_t m, int64_t p, int *bn, int *bk,
                        int *stages, int *group_m);

/* Tail split the split path would use for one product n x m x p (mm_gemm,
 * or a grouped call holding only this product) on the current device:
 * *tiles = number of 128 x bn output tiles; tiles *split_from .. *tiles - 1,
 * the last, partly filled wave of the persistent grid, each run as *split_s
 * parts along K whose FP32 partial tiles the part finishing last adds in part
 * order (*split_s = 1, *split_from = *tiles: no split).  Grouped calls of
 * several products and the allocation-free entry point do not split.
 * Needs mm_init (the SM count); any pointer may be NULL. */
mm_status mm_tune_query_tail(int64_t n, int64_t m, int64_t p, int *tiles,
                             int *split_from, int *split_s);

/* Fused split-K plan of the split path for one product n x m x p (mm_gemm /
 * mm_gemm_async on MM_MODE_SPLIT_BF16X3 or _X6): a product with fewer
 * 128 x 128 output tiles than half the SMs, whose slices need at most eight
 * 64-wide K blocks each, with A and B 16-byte aligned and m and p multiples
 * of 4 (the kernel loads them with TMA), runs as ONE launch that reads A and B
 * directly, splits each 64-wide K block into bf16 parts in shared memory
 * (power-of-two scales per row of A and column of B within a block, only for
 * blocks holding an entry outside [2^-40, 2^40]), multiplies on the tensor
 * cores and adds the blocks' FP32 partial products in registers; the inner
 * dimension of each tile is cut into *slices slices, one CTA each, in
 * *clusters thread-block clusters of *cluster_size CTAs that add their
 * partial tiles through distributed shared memory (and, for *clusters > 1,
 * through library scratch, the cluster finishing last adding the others in
 * order).  The result does not depend on timing.  *slices = 0: the product
 * takes the packed path (mm_tune_query_tail).  Grouped calls and serving
 * batches always take the packed path, so a product's bits there equal a
 * grouped call of that product alone; against mm_gemm they agree within the
 * split path's tolerance.  Needs mm_init; any pointer may be NULL. */
mm_status mm_tune_query_splitk(int64_t n, int64_t m, int64_t p, int *tiles, int *slices,
                               int *clusters, int *cluster_size);

/* K-slice plan of a SIMT (dt = MM_F32) or DGEMM (dt = MM_F64) product, a
 * pure host function (no device, no mm_init): the plan mm_gemm follows on a
 * device of `sms` SMs (sms <= 0: the initialised device's count, 148 before
 * mm_init).  A product with fewer whole output tiles (128 x 128 in FP32,
 * 64 x 64 in FP64) than half the SMs is cut along K into *slices slices of
 * *slice_k values (the last one shorter), computed on *tile x *tile output
 * tiles (64, or 128 for FP32 products at least 128 wide both ways); the
 * slices' partial sums are then added in a fixed order.  The plan keeps one
 * wave of at most two CTAs per SM, slices of at least 128 values unless K is
 * shorter, and partials of at most 256 MiB; it depends on the shape (and
 * sms) only and is the same for (n, m, p) and (p, m, n).  *slices = 0: the
 * one-pass kernel (*tile its tile, *slice_k 0).  Returns MM_EINVAL for
 * negative sizes, another dtype or NULL outputs.  Not in the paper. */
mm_status mm_simt_plan(int64_t n, int64_t m, int64_t p, mm_dtype dt, int sms, int *slices,
                       int64_t *slice_k, int *tile);

/* The tail-split planner itself, a pure host function (no device, no
 * mm_init): for a product of `tiles` output tiles of 128 x bn, kt pack rows
 * of K (64 bf16 or 128 e4m3 values each), inner dimension m and `products`
 * bf16 products per K step (3 or 6 for the split kinds, 0.5 for e4m3) on
 * `grid` persistent CTAs, writes the first split tile and the number of K
 * parts (1: no split).  It picks the split that minimises a makespan model of
 * the round-robin assignment of work units to CTAs: at most 4 parts, at
 * least 2 pack rows per part, at most 2 x grid split units, and no split for
 * products with fewer tiles than CTAs and fewer than 16 pack rows.
 * Returns MM_EINVAL for negative sizes or NULL outputs. */
mm_status mm_tail_plan(int64_t tiles, int grid, int kt, int bn, int64_t m,
                       double products, int *split_from, int *split_s);

/* Measured fused multiply-add rate of the CUDA cores for dtype dt (FP32
 * FFMA or FP64 DFMA), in flops per second (2 per FMA): a grid of several
 * blocks per SM runs independent FMA chains on registers for `iters` rounds
 * of 192 FMAs per thread, timed with CUDA events on the library stream.  The
 * denominator of the SIMT FP32 and DGEMM kernels' rooflines; it reads the
 * device only.  Synchronous.  Not in the paper. */
mm_status mm_measure_fma_peak(mm_dtype dt, int64_t iters, double *flops_per_s);

/* ----------------------------------------------------------------- tracing */

/* When enabled, every kernel the library launches is bracketed by CUDA events
 * on its stream; mm_trace_read returns the launch count and summed device
 * time (ms) of the kernel named `kernel` ("simt_f32", "dgemm_f64", "simt_sum" (the
 * fixed-order sum of a K-sliced SIMT or FP64 product), "split_maps", "split_pack",
 * "split_verify", "split_fix", "split_tc", "fused_tc", "fp8_max", "fp8_pack", "fp8_tc",
 * "fp8_blk", "check_f64", "ozaki_max", "ozaki_map", "ozaki_digits", "ozaki_sum",
 * "ozaki_gate", "add", "diag", "cplx_planes", "cplx_combine") since the last reset.
 * Reading synchronises the recorded events. */
mm_status mm_trace_enable(int on);
mm_status mm_trace_reset(void);
mm_status mm_trace_read(const char *kernel, int64_t *launches, double *total_ms);

/* Number of library kernel launches since mm_init (all kernels). */
int64_t mm_launch_count(void);

/* ------------------------------------------- related products of the paper */

/* Complex C = A.B for complex64 matrices (interleaved re, im; row-major,
 * dense): the product of the paper's Table 2 "complex float" column.  Runs
 * the four real products Ar.Br, Ai.Bi, Ar.Bi, Ai.Br as one grouped call of the
 * chosen real path (MM_MODE_SIMT or MM_MODE_SPLIT_BF16X3; AUTO = split) and
 * assembles C.  Device pointers; synchronous; library scratch holds the
 * planes and partial products.  Accuracy: max |c^ - c| / sum_r |a_ir||b_rj|
 * <= 2e-6 sqrt(m) (moduli). */
mm_status mm_cgemm(int64_t n, int64_t m, int64_t p, const void *A, const void *B,
                   void *C, mm_mode mode);

/* C = alpha A + beta B elementwise for n x p matrices (device pointers, dtype
 * dt): the matrix addition / subtraction the paper measures beside the
 * product (results section).  alpha = 1, beta = +-1 give one correctly
 * rounded addition or subtraction per entry; otherwise fma(alpha, a, beta b).
 * Synchronous. */
mm_status mm_add(int64_t n, int64_t p, double alpha, const void *A, double beta,
                 const void *B, void *C, mm_dtype dt);

/* Product with a diagonal matrix, the special case the paper names in its
 * algorithms section: side 0: C = X.diag(d) (c_ij = x_ij d_j, d has p
 * entries); side 1: C = diag(d).X (c_ij = d_i x_ij, d has n entries).  One
 * correctly rounded product per entry; reads X once.  X, C: n x p, device
 * pointers, dtype dt.  Synchronous. */
mm_status mm_diag(int64_t n, int64_t p, const void *X, const void *d, void *C,
                  int side, mm_dtype dt);

/* Asynchronous forms of mm_add and mm_diag: the same arguments plus `stream`
 * (a cudaStream_t; NULL = the library stream).  They validate the arguments,
 * queue the kernel and return; C is complete when the stream reaches that
 * point (mm_sync(stream), or any later work on the stream).  A failure of
 * the kernel itself shows at the next synchronising call. */
mm_status mm_add_async(int64_t n, int64_t p, double alpha, const void *A, double beta,
                       const void *B, void *C, mm_dtype dt, void *stream);
mm_status mm_diag_async(int64_t n, int64_t p, const void *X, const void *d, void *C,
                        int side, mm_dtype dt, void *stream);

/* ------------------------------------------------ allocation-free variant */

/* The FP32 split product of mm_gemm's MM_MODE_SPLIT_BF16X3 path, for callers
 * that must not allocate device memory: a plug-in running inside a host
 * framework that owns and accounts for all device memory, code on a latency-
 * critical path where cudaMalloc's implicit synchronisation is not
 * acceptable, or a process whose device memory budget is fixed at start-up.
 * The paper has no counterpart to this entry point.
 *
 * Scratch: the scale words, problem table, packed bf16 operands and timeout
 * flag of the split path live in one fixed 64 MiB device array compiled into
 * the library (every GPU that loads the library holds it until the process
 * exits).  The call makes no cudaMalloc, cudaFree or other allocating call and
 * does not need mm_init.  Products whose scratch does not fit are rejected
 * with MM_ESCRATCH (2048^3 fits, 3072^3 does not).
 * A (n x m), B (m x p), C (n x p): device pointers, FP32, row-major and dense
 * as in mm_gemm.  stream: a cudaStream_t (NULL: the legacy default stream);
 * the call synchronises that stream and returns when C is written.  Same kernels and tile choices as
 * mm_gemm's split path, without its tail split (mm_tune_query_tail): where
 * mm_gemm splits tiles along K the two results differ only in the rounding
 * of that one extra addition, within the split path's tolerance; elsewhere
 * they are identical.
 * Every call uses the same array, which keeps the previous call's contents
 * (the call clears what must start at zero): calls whose work overlaps on the
 * GPU - on different streams or from different host threads - race and
 * corrupt each other; serialise them.  The first call on a device looks up
 * the array's device address on that device (with it current); make that
 * first call before any stream capture.  Returns MM_OK, MM_EINVAL,
 * MM_ESCRATCH, MM_EUNSUPPORTED (not an sm_103 device), MM_ETIMEOUT (a
 * device-side wait ran out) or MM_ECUDA. */
mm_status mm_gemm_split_static(int64_t n, int64_t m, int64_t p, const float *A,
                               const float *B, float *C, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MM_H */
