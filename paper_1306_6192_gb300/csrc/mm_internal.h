// Internal declarations shared by the library's translation units.
// Not part of the public ABI (include/mm.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/mm.h"

namespace mm {

// ------------------------------------------------------------ tile constants
// SIMT FP32 tile (the shared-memory tiling of the paper's Listing 4, scaled up
// with register blocking): 128 x 128 outputs per 256-thread block, 8 x 8 per
// thread, k-slices of 16.
constexpr int kSimtF32BM = 128, kSimtF32BN = 128, kSimtF32BK = 16;
// SIMT FP64 tile: 64 x 64 outputs per 256-thread block, 4 x 4 per thread.
constexpr int kSimtF64BM = 64, kSimtF64BN = 64, kSimtF64BK = 8;

// Tensor-core paths (split-BF16x3 and e4m3): the M tile is the tcgen05 M
// (128 rows of A).  Packed operands live in the scratch "pack region", viewed
// as rows of 128 bytes: one pack row holds one K block of one row of A (or
// one column of B) - 64 bf16 values for the split path, 128 e4m3 values for
// the FP8 path.
constexpr int kTcBM = 128;
constexpr int kPackRowBytes = 128;
// Split kinds: two bf16 parts (hi, lo; products hi.hi + hi.lo + lo.hi) or
// three (hi, mid, lo; the six products down to 2^-16 relative).
enum TcKind : int { kTcSplitBf16x3 = 0, kTcE4m3 = 1, kTcSplitBf16x6 = 2 };
// elements per pack row and operand parts
inline int pack_k(TcKind k) { return k == kTcE4m3 ? 128 : 64; }
inline int pack_parts(TcKind k) { return k == kTcE4m3 ? 1 : (k == kTcSplitBf16x3 ? 2 : 3); }
constexpr int kPackK = 64;  // bf16 elements per pack row

// ------------------------------------------------------------ epilogue
// C = alpha (A.B) + beta D of one product (mm_gemm_axpby), applied by the
// kernel that writes C, to the product x of entry (i, j): on = 0 writes x,
// on = 1 alpha x, on = 2 fma(alpha, x, beta d) with d = D[i p + j] (D is n x p
// row-major like C; it may be C itself, since each entry of C is read and
// written by the same thread).  Zero-initialised: off.
template <typename T>
struct EpiT {
  const T *D;
  T alpha, beta;
  int on;
};
using EpiF = EpiT<float>;
#ifdef __CUDACC__
template <typename T>
__device__ __forceinline__ T epi_apply(const EpiT<T> &e, T x, int64_t idx) {
  if (e.on == 0) return x;
  if (e.on == 1) return e.alpha * x;
  return fma(e.alpha, x, e.beta * e.D[idx]);
}
#endif
// The host request: alpha and beta as given (rounded to T for the kernels),
// D a device pointer or null where beta == 0.
struct Epi {
  double alpha, beta;
  const void *D;
  template <typename T>
  EpiT<T> as() const {
    EpiT<T> e{static_cast<const T *>(D), (T)alpha, (T)beta, 0};
    e.on = e.beta != T(0) ? 2 : (e.alpha != T(1) ? 1 : 0);
    if (e.on != 2) e.D = nullptr;
    return e;
  }
};
template <typename T>
inline EpiT<T> epi_of(const Epi *e) {
  return e ? e->as<T>() : EpiT<T>{nullptr, T(1), T(0), 0};
}

// ------------------------------------------------------------ device tables
// One product of a tensor-core path, as the prep and tensor-core kernels see
// it.  With P = pack_parts(kind) and kt = ceil(m / pack_k(kind)):
//   A pack tile (mt, kb): rows a_row0 + (mt*kt + kb)*P*128 ..:
//       part 0 (split: hi; FP8: the e4m3 values) of A rows mt*128 .. +127 for
//       K block kb, then part 1 (split: lo) in the next 128 rows;
//   B pack tile (nt, kb): rows b_row0 + (nt*kt + kb)*P*bn ..:
//       part 0 of B columns nt*bn .. +bn-1 (B transposed so K is contiguous),
//       then part 1 in the next bn rows.
// Entries outside A or B are zero.  sA[i] / tB[j] hold the bit pattern of
// max_r |a_ir| / max_r |b_rj|; each path derives its power-of-two scale
// exponent of a row/column from it.
// Tail split (a property of the product's own shape, see tc_tail_plan): its
// tiles split_from .. mt*nt-1 in raster order run as split_s parts along K
// (part h: pack rows [h*kt/split_s, (h+1)*kt/split_s)); part h of split tile
// t writes its FP32 partial tile to part + ((t - split_from)*split_s + h) *
// 128*bn ([column][row] order) and counts itself in cnt[t - split_from]
// (zero before the launch); the last part adds the parts in order 0, 1, ...
// The tensor-core kernel's work units of the product: split_from whole tiles,
// then the parts; unit_start is their prefix over the problems of a table.
struct SplitProb {
  const float *A;
  const float *B;
  float *C;
  int64_t a_row0, b_row0;
  uint32_t *sA, *tB;
  // split kinds: max |x| per (K block, row of A) and (K block, column of B),
  // written by the unscaled pack: pA[kb*n + i], pB[kb*p + j]
  uint32_t *pA, *pB;
  int32_t n, m, p;
  int32_t mt, nt, kt;      // ceil(n/128), ceil(p/bn), ceil(m/pack_k)
  int32_t bn, group_m;     // N tile (64, 128 or 256), raster band height
  int32_t unit_start;      // prefix over problems of tensor-core work units
  int32_t pack_start;      // prefix of pack tiles: mt*kt + nt*kt
  int32_t ver_start;       // prefix of verify items: ceil((n + p) / 32) each
  int32_t split_from;      // tail split (split_s <= 1: none; then split_from
  int32_t split_s;         //   is ignored and every tile is one unit)
  float *part;             // partial tiles of the split tiles
  int *cnt;                // parts finished per split tile
  // pack tiles between consecutive row tiles of A / column tiles of B (0:
  // kt, the layout above); a larger stride lets a product read a window of
  // kt K blocks out of a longer pack (the FP64 emulation's level products)
  int32_t a_kstride, b_kstride;
  // 1 + index of C's tensor map in the launch's map array (tiled stores of
  // the epilogue); 0: C is written with plain stores
  int32_t c_tma;
  // C = alpha (A.B) + beta D (plain stores only; off: C = A.B)
  EpiF epi;
};

// Work units of a product with its tail split: whole tiles, then the parts.
__host__ __device__ inline int64_t split_units(const SplitProb &sp) {
  const int64_t tiles = (int64_t)sp.mt * sp.nt;
  return sp.split_s > 1 ? sp.split_from + (tiles - sp.split_from) * sp.split_s : tiles;
}

// One product of the fused split-K path (tc_fused.cu): output tiles of
// 128 x 128 in row-major tile order, each tile's K blocks of 64 cut into S
// slices [h*kb/S, (h+1)*kb/S), one CTA per slice, S = Q * CS with CS the
// launch's cluster size.  With Q > 1 the clusters of a tile meet through
// `slots` (tiles * Q partial tiles of 128 x 128 floats) and `cnt` (tiles * CS
// counters, zero between launches).
struct FusedProb {
  const float *A;
  const float *B;
  float *C;
  int32_t n, m, p;
  int32_t mt, nt, kb;      // ceil(n/128), ceil(p/128), ceil(m/64)
  int32_t S, Q;            // slices per tile, clusters per tile
  float *slots;
  int *cnt;
  EpiF epi;  // C = alpha (A.B) + beta D (off: C = A.B)
};

// One product of the grouped SIMT path (f32 or f64 elements).
struct SimtProb {
  const void *A;
  const void *B;
  void *C;
  int64_t n, m, p;
  int32_t tiles_n;     // tiles along p
  int32_t tile_start;  // prefix over problems of tiles
};

// ------------------------------------------------------------ launchers
// epi (null: C = A.B) as for EpiT, applied where C is written.
cudaError_t launch_simt_f32(int64_t n, int64_t m, int64_t p, const float *A,
                            const float *B, float *C, cudaStream_t s, const Epi *epi = nullptr);
// run_if: a device word; when given, the product runs only if it is non-zero
// when the kernel starts (the FP64 emulation's fallback).
cudaError_t launch_simt_f64(int64_t n, int64_t m, int64_t p, const double *A,
                            const double *B, double *C, cudaStream_t s,
                            const int *run_if = nullptr, const Epi *epi = nullptr);
cudaError_t launch_simt_grouped(bool f64, const SimtProb *d_probs, int nprobs,
                                int total_tiles, bool all_vec, cudaStream_t s);
// Split-K of a SIMT product with too few output tiles for the SMs: S slices
// of ks K values (S = 0: the one-pass kernel) on 64 x 64 tiles, or 128 x 128
// (wide: FP32 products at least 128 wide both ways), from the product's shape
// alone.  With S > 1 the slices' partials go to `part` (S n p elements) and a
// second kernel adds them into C in a fixed order.
struct SimtPlan {
  int S;
  int64_t ks;
  bool wide;
};
SimtPlan simt_plan(bool f64, int64_t n, int64_t m, int64_t p);
// The same plan for a device of `sms` SMs (host only; mm_simt_plan).
SimtPlan simt_plan_for(bool f64, int64_t n, int64_t m, int64_t p, int sms);
size_t simt_scratch_bytes(bool f64, int64_t n, int64_t m, int64_t p);
cudaError_t launch_simt_splitk_f32(int64_t n, int64_t m, int64_t p, const float *A, const float *B,
                                   float *C, float *part, const SimtPlan &pl, cudaStream_t s,
                                   const Epi *epi = nullptr);
// run_if: as for launch_simt_f64 (the FP64 emulation's fallback).
cudaError_t launch_simt_splitk_f64(int64_t n, int64_t m, int64_t p, const double *A,
                                   const double *B, double *C, double *part, const SimtPlan &pl,
                                   cudaStream_t s, const int *run_if = nullptr,
                                   const Epi *epi = nullptr);

// Prep of the packed split path: the split (hi/lo bf16) into the packs with
// the row/column maxima, their verification and the re-pack of operands out
// of range.
// `map` arguments: item -> problem index arrays written by
// launch_split_maps for tables of several problems, or nullptr.
cudaError_t launch_split_maps(const SplitProb *d_probs, int nprobs, int *unit_map,
                              int *pack_map, int *ver_map, cudaStream_t s);
// Verify items of a product: 32 rows/columns each.
__host__ __device__ inline int64_t verify_items(int64_t n, int64_t p) { return (n + p + 31) / 32; }
// Pack modes (split kinds) and the per-problem flags they use.
constexpr int kPackUnscaled = 1, kPackFix = 2;
constexpr int kFlagScaleA = 1, kFlagScaleB = 2;
// kPackUnscaled: one block per pack tile.  kPackFix: a persistent grid that
// returns at once unless *any is set, then re-packs the tiles of flagged
// operands (flags[g]).
cudaError_t launch_split_pack(TcKind kind, int mode, const SplitProb *d_probs, int nprobs,
                              int total_tiles, const int *map, const int *flags, const int *any,
                              void *pack_base, cudaStream_t s);
// After an unscaled pack: reduces the partial maxima into sA / tB and sets
// flags[g] (and *any) for operands out of range; flags and *any zeroed by
// the caller.  total_items = sum over problems of verify_items(n, p); map:
// item -> problem (tables of several problems) or nullptr; max_kt = the
// largest kt of the table.  write_cols = false leaves tB as it is (a later
// slab sharing B's words, which another stream may be reading) but still
// flags B.
cudaError_t launch_split_verify(const SplitProb *d_probs, int nprobs, int64_t total_items,
                                const int *map, int *flags, int *any, int max_kt, cudaStream_t s,
                                bool write_cols = true);
// Tensor-core mainloop + epilogue over all work units of all problems.
struct TcConfig {
  int bkb;      // bytes of K per pipeline stage and pack row: 64 or 128
  int stages;   // pipeline depth (tables with max_bn > 128)
  int grid;     // persistent CTAs (<= number of SMs; 0 = one per SM)
  int max_bn = 256;  // widest N tile of the table: <= 128 selects the deeper
                     // rings of the 128-wide layouts
};
int tc_grid(const TcConfig &cfg);
// Tail-split plan of one product from its own shape only (so that a product
// gets the same split, hence the same bits, alone and in any grouped table):
// `tiles` output tiles of 128 x bn, kt pack rows of K, the kind's bf16 (or
// e4m3) products per K step, on `grid` persistent CTAs.  The makespan model
// of the product run alone decides; a product that fills less than one wave
// and has fewer than 16 pack rows is never split (grouped tables of many
// small products gain nothing from it).
struct TcTail {
  int split_from, split_s;
};
TcTail tc_tail_plan(int64_t tiles, int grid, int kt, int bn, int64_t m, double products);
// Scratch of a plan: partial tiles (256-byte aligned), then the counters.
size_t tc_tail_bytes(const TcTail &t, int64_t tiles, int bn);
size_t tc_tail_part_bytes(const TcTail &t, int64_t tiles, int bn);
// flags: per-problem kFlagScaleA / kFlagScaleB (nullptr: both operands were
// packed scaled).  order: the work units of each CTA (tc_unit_order, on the
// device), or nullptr for units c, c + grid, c + 2 grid, ... on CTA c.
// uniform_only (FP8 with per-block factors): only the tiles whose rows and
// columns keep one exponent along K (flags in each problem's cnt) run.
cudaError_t launch_tc(TcKind kind, const SplitProb *d_probs, int nprobs,
                      int total_units, const int *unit_map, const int *flags,
                      void *pack_base, int64_t pack_rows, const TcConfig &cfg,
                      int *d_err, cudaStream_t s, const int *order = nullptr,
                      int uniform_only = 0, const void *c_maps = nullptr);
// Tensor map over C for the tensor-core epilogue's tiled stores (128 bytes
// written to `map`); usable where tc_c_map_ok holds.
bool tc_c_map_ok(const float *C, int64_t n, int64_t p);
cudaError_t encode_c_map(void *map, float *C, int64_t n, int64_t p);
// CTAs of a tensor-core launch of total_units work units.
int tc_launch_grid(const TcConfig &cfg, int64_t total_units);
// Work units per CTA for a table whose units differ in length (a grouped
// table, the FP64 emulation's levels): each unit, in index order, goes to the
// CTA the cost model (K pack rows of the unit, plus one for its fixed cost)
// expects to be free first, the lowest-numbered CTA on a tie.  The CTAs then
// work on neighbouring units at any time, so the operand tiles that
// neighbouring units share are still in L2 when the second one reads them, and
// they finish together; with units of equal length the schedule is the
// round-robin one.  out: grid + 1 offsets into the list that follows, then the
// units of CTA 0, of CTA 1, ... (each ascending).  Host only.
void tc_unit_order(const SplitProb *tab, int nprobs, int grid, std::vector<int> &out);

// Fused split-K launch of one product (tiles * S CTAs in clusters of cs =
// S / Q); six: three bf16 parts.  The operands are read by TMA, so A and B
// must be 16-byte aligned with m and p multiples of 4 (fused_operands_ok).
bool fused_operands_ok(const float *A, const float *B, int64_t m, int64_t p);
cudaError_t launch_fused(bool six, const FusedProb &pr, int cs, int *d_err, cudaStream_t s);
// Most CTAs of the fused kernel resident at once with clusters of cs CTAs
// (cs = 1, 2, 4, 8), measured once per device and kind.
int fused_capacity(bool six, int cs);

// FP64 check (Freivalds + sampled entries): writes 2 doubles to d_out.
cudaError_t launch_check(bool f64, int64_t n, int64_t m, int64_t p,
                         const void *A, const void *B, const void *C,
                         const double *x, int64_t nsamples, const int64_t *I,
                         const int64_t *J, double *d_work, double *d_out,
                         cudaStream_t s);
size_t check_work_doubles(int64_t n, int64_t m, int64_t p);

// ------------------------------------------------------------ tracing
// Brackets a launch with events when tracing is on; counts every launch.
void trace_begin(const char *name, cudaStream_t s);
void trace_end(const char *name, cudaStream_t s);
void trace_clear();

struct TraceScope {
  const char *name;
  cudaStream_t s;
  TraceScope(const char *n, cudaStream_t st) : name(n), s(st) { trace_begin(n, st); }
  ~TraceScope() { trace_end(name, s); }
};

int sm_count();

// Status from a CUDA error code.
mm_status from_cuda(cudaError_t e);

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace mm
