// FP8 (e4m3) product with per-block power-of-two scales (MM_MODE_FP8).
//
// Scales: each row of A and each column of B is cut into K blocks of 128
// values; every (row, block) of A and (block, column) of B gets its own
// power of two 2^-e that brings the block's largest magnitude into [128, 256)
// (below the e4m3 maximum 448), and its 128 values are rounded to e4m3 (round
// to nearest even, saturating).  Finer scales than one per row keep more of
// the significance of blocks whose values are far below the row's largest.
//
// Kernels:
//   fp8blk_pack_kernel  one block per pack tile (128 rows of A, or 256
//                       columns of B, by one K block): the block's row /
//                       column maxima, the factors 2^e (per row or column
//                       and K block, padded to whole tiles), block 0's maxima
//                       as the row / column scale words, and the e4m3 pack
//                       rows (the layout of mm_internal.h, bn = 256).
//   fp8blk_flag_kernel  per row tile of A and 128-column sub-tile of B: 1
//                       when every row (column) has the same exponent in all
//                       K blocks.
//   tc_gemm_kernel      (tc_gemm.cu, e4m3, 128 x 256 tiles) the tiles whose
//                       row tile and both column sub-tiles are flagged: all
//                       K blocks accumulated in tensor memory, one factor per
//                       row and column applied in the epilogue; it skips the
//                       other tiles.
//   fp8blk_gemm_kernel  the other tiles, as 128 x 128 sub-tiles; persistent,
//                       warp-specialised: a TMA producer (pack
//                       tiles of each K block into a shared-memory ring, and
//                       the block's exponents into a second ring), one thread
//                       issuing four tcgen05.mma kind::f8f6f4 per K block
//                       into one of four 128-column tensor-memory
//                       accumulators, and eight worker warps that load each
//                       block's FP32 partial product (tcgen05.ld), multiply it
//                       by 2^(e_i + e_j) exactly and add it into registers,
//                       then store the tile.  The K blocks are added in order
//                       with round-to-nearest FP32 additions.  A tile whose
//                       rows and columns keep one exponent along K (flagged
//                       by fp8blk_flag_kernel) accumulates all its blocks in
//                       one accumulator instead and is unscaled once.
// The error of the result against the FP64 oracle is measured and reported;
// there is no tolerance for it.  The product is the paper's (Section
// "Implementacje algorytmow"); the FP8 path is this library's, not the
// paper's.  Every mbarrier wait is bounded (device flag, MM_ETIMEOUT).
#include <cuda_fp8.h>
#include <cudaTypedefs.h>

#include <cstring>

#include "ctx.h"
#include "tc_ptx.cuh"

namespace mm {
namespace {

using namespace tcx;

constexpr int kBK = 128;              // e4m3 values per K block (one pack row)
constexpr int kBN = 128;              // N tile of the blockwise kernel
constexpr int kPackBN = 256;          // columns of B per pack tile (two kBN sub-tiles)
constexpr int kStages = 6;            // operand ring
constexpr int kEStages = 8;           // scale-factor ring
constexpr int kAccs = 4;              // 128-column accumulators in 512 columns
constexpr int kWorkers = 256;         // warps 2..9: two per TMEM lane quarter
constexpr int kWCols = kBN * 128 / kWorkers;  // accumulator columns per worker thread
constexpr int kThreads = 64 + kWorkers;
constexpr uint64_t kWaitNs = 4000000000ull;
constexpr uint64_t kDrainNs = 200000000ull;

struct Lay {
  static constexpr int kA = kTcBM * kBK;                  // 16 KB
  static constexpr int kB = kBN * kBK;                    // 16 KB
  static constexpr int kStage = kA + kB;
  static constexpr int kEOff = kStages * kStage;          // factors: 128 + 128 floats
  static constexpr int kESlot = 2 * 128 * 4;
  static constexpr int kBarOff = kEOff + kEStages * kESlot;
  // full[S], empty[S], efull[E], eempty[E], acc_full[A], acc_empty[A], drain
  static constexpr int kNumBars = 2 * kStages + 2 * kEStages + 2 * kAccs + 1;
  static constexpr int kMiscOff = kBarOff + kNumBars * 8;
  static constexpr int kSmem = kMiscOff + 64 + 1024;
};
static_assert(Lay::kSmem <= 232448, "shared memory budget");

// Exponent of a block whose largest magnitude has bit pattern max_bits: the
// scaled maximum lies in [128, 256); 0 for an all-zero or non-finite block.
__device__ __forceinline__ int blk_exponent(uint32_t max_bits) {
  const float f = __uint_as_float(max_bits);
  return (f > 0.0f && f <= 3.402823466e38f) ? scale_exponent(max_bits) - 7 : 0;
}

// Exponent of a block: its own, or the whole row's (column's) when the
// block's largest magnitude lies within one binade of the row's (an all-zero
// block too), so that the blocks of rows without a wide spread of magnitudes
// share one factor and their tiles can be accumulated along K in tensor
// memory; a block two or more binades below keeps its own.  Rows with a NaN
// or an infinity keep the blocks' own exponents.
__device__ __forceinline__ int pick_exponent(uint32_t blk_max, uint32_t whole_max) {
  const int eb = blk_exponent(blk_max);
  if (!(__uint_as_float(whole_max) <= 3.402823466e38f)) return eb;
  const int ew = blk_exponent(whole_max);
  return (blk_max == 0 || eb >= ew - 1) ? ew : eb;
}

__device__ __forceinline__ uint32_t to_e4m3x4(float4 x, int e) {
  const __nv_fp8x2_storage_t lo = __nv_cvt_float2_to_fp8x2(
      make_float2(scale_pow2(x.x, -e), scale_pow2(x.y, -e)), __NV_SATFINITE, __NV_E4M3);
  const __nv_fp8x2_storage_t hi = __nv_cvt_float2_to_fp8x2(
      make_float2(scale_pow2(x.z, -e), scale_pow2(x.w, -e)), __NV_SATFINITE, __NV_E4M3);
  return (uint32_t)lo | ((uint32_t)hi << 16);
}

__device__ __forceinline__ uint32_t absb(float x) { return __float_as_uint(x) & 0x7fffffffu; }

__device__ __forceinline__ bool al16(const void *p) {
  return (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
}

// Scale factors of a problem (pA / pB of its SplitProb): 2^e per row of A and
// K block, [kt][mt * 128], and per K block and column of B, [kt][nt * 128],
// as floats (2^e is exact for e >= -149).
__device__ __forceinline__ float *fac_a(const SplitProb &pr) { return reinterpret_cast<float *>(pr.pA); }
__device__ __forceinline__ float *fac_b(const SplitProb &pr) { return reinterpret_cast<float *>(pr.pB); }

__device__ __forceinline__ float pow2f(int e) { return scale_pow2(1.0f, e); }

// Whole-row maxima of A and whole-column maxima of B (bit patterns of |x|,
// which order like the magnitudes) into the problem's sA / tB (zeroed before
// the launch).  Items of a problem, from the prefix `split_from` of its entry
// in the blockwise table: ceil(n / 8) items of 8 rows of A (a warp per row,
// 16-byte loads where the row allows), then strips of 128 columns x 256 rows
// of B (four columns per lane), merged with atomicMax.
constexpr int kMaxRows = 8, kMaxStrip = 128, kMaxChunk = 256;

__host__ __device__ inline int64_t max_items(int64_t n, int64_t m, int64_t p) {
  return (n + kMaxRows - 1) / kMaxRows +
         ((p + kMaxStrip - 1) / kMaxStrip) * ((m + kMaxChunk - 1) / kMaxChunk);
}

__device__ __forceinline__ uint32_t absmax4(float4 v) {
  return max(max(__float_as_uint(v.x) & 0x7fffffffu, __float_as_uint(v.y) & 0x7fffffffu),
             max(__float_as_uint(v.z) & 0x7fffffffu, __float_as_uint(v.w) & 0x7fffffffu));
}

__global__ void __launch_bounds__(256)
fp8blk_max_kernel(const SplitProb *__restrict__ probs, int nprobs) {
  const int item = blockIdx.x;
  const int g =
      find_problem(probs, nprobs, nullptr, item, [](const SplitProb &q) { return q.split_from; });
  const SplitProb &pr = probs[g];
  const int64_t local = item - pr.split_from;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t items_a = (pr.n + kMaxRows - 1) / kMaxRows;
  if (local < items_a) {
    const int64_t i = local * kMaxRows + warp;
    if (i >= pr.n) return;
    const float *row = pr.A + i * pr.m;
    uint32_t mx = 0;
    if ((reinterpret_cast<uintptr_t>(pr.A) & 15u) == 0 && (pr.m & 3) == 0) {
      const float4 *r4 = reinterpret_cast<const float4 *>(row);
      for (int64_t k = lane; k < pr.m / 4; k += 32) mx = max(mx, absmax4(__ldg(r4 + k)));
    } else {
      for (int64_t k = lane; k < pr.m; k += 32) mx = max(mx, __float_as_uint(row[k]) & 0x7fffffffu);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) pr.sA[i] = mx;
    return;
  }
  __shared__ uint32_t part[8][kMaxStrip];
  const int64_t b = local - items_a;
  const int64_t strips = (pr.p + kMaxStrip - 1) / kMaxStrip;
  const int64_t c0 = (b % strips) * kMaxStrip + 4 * lane, r0 = (b / strips) * kMaxChunk;
  const bool vec = (reinterpret_cast<uintptr_t>(pr.B) & 15u) == 0 && (pr.p & 3) == 0;
  uint32_t mx[4] = {0, 0, 0, 0};
  for (int r = warp; r < kMaxChunk; r += 8) {
    const int64_t k = r0 + r;
    if (k >= pr.m) break;
    const float *src = pr.B + k * pr.p + c0;
    if (vec && c0 + 4 <= pr.p) {
      const float4 v = __ldg(reinterpret_cast<const float4 *>(src));
      mx[0] = max(mx[0], __float_as_uint(v.x) & 0x7fffffffu);
      mx[1] = max(mx[1], __float_as_uint(v.y) & 0x7fffffffu);
      mx[2] = max(mx[2], __float_as_uint(v.z) & 0x7fffffffu);
      mx[3] = max(mx[3], __float_as_uint(v.w) & 0x7fffffffu);
    } else {
#pragma unroll
      for (int e = 0; e < 4; e++)
        if (c0 + e < pr.p) mx[e] = max(mx[e], __float_as_uint(src[e]) & 0x7fffffffu);
    }
  }
#pragma unroll
  for (int e = 0; e < 4; e++) part[warp][4 * lane + e] = mx[e];
  __syncthreads();
  if (threadIdx.x < kMaxStrip) {
    uint32_t v = 0;
#pragma unroll
    for (int w = 0; w < 8; w++) v = max(v, part[w][threadIdx.x]);
    const int64_t col = (b % strips) * kMaxStrip + threadIdx.x;
    if (col < pr.p) atomicMax(&pr.tB[col], v);
  }
}

__global__ void __launch_bounds__(256)
fp8blk_pack_kernel(const SplitProb *__restrict__ probs, int nprobs, const int *__restrict__ map,
                   uint32_t *__restrict__ pack) {
  constexpr int kQuads = kBK / 4;  // 32-bit words per pack row
  __shared__ float tile[kBK][64 + 1];
  __shared__ int colexp[64];
  __shared__ uint32_t colmax[4][64];
  const int item = blockIdx.x;
  const int g =
      find_problem(probs, nprobs, map, item, [](const SplitProb &q) { return q.pack_start; });
  const SplitProb &pr = probs[g];
  const int local = item - pr.pack_start;
  const int tid = threadIdx.x, lane = tid & 31;
  if (local < pr.mt * pr.kt) {
    // A tile (mt, kb): rows mt*128 + tid/32 + 8 it, a warp per row, four
    // values per lane
    const int mt = local / pr.kt, kb = local % pr.kt;
    const int64_t base = pr.a_row0 + (int64_t)local * kTcBM;
    const bool vec = al16(pr.A) && (pr.m & 3) == 0;
    float4 xs[16];
#pragma unroll
    for (int it = 0; it < 16; it++) {
      const int r = (tid >> 5) + 8 * it;
      const int64_t i = (int64_t)mt * kTcBM + r;
      const int64_t k = (int64_t)kb * kBK + 4 * lane;
      float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
      if (i < pr.n) {
        const float *row = pr.A + i * pr.m;
        if (vec && k + 4 <= pr.m) {
          x = __ldcs(reinterpret_cast<const float4 *>(row + k));
        } else {
          if (k < pr.m) x.x = row[k];
          if (k + 1 < pr.m) x.y = row[k + 1];
          if (k + 2 < pr.m) x.z = row[k + 2];
          if (k + 3 < pr.m) x.w = row[k + 3];
        }
      }
      xs[it] = x;
    }
#pragma unroll
    for (int it = 0; it < 16; it++) {
      const int r = (tid >> 5) + 8 * it;
      uint32_t mx = max(max(absb(xs[it].x), absb(xs[it].y)), max(absb(xs[it].z), absb(xs[it].w)));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      const int e = pick_exponent(mx, pr.sA[(int64_t)mt * kTcBM + r]);
      if (lane == 0) fac_a(pr)[(int64_t)kb * pr.mt * kTcBM + (int64_t)mt * kTcBM + r] = pow2f(e);
      pack[(base + r) * kQuads + lane] = to_e4m3x4(xs[it], e);
    }
  } else {
    // B tile (nt, kb): 256 columns x 128 k, transposed through shared memory
    // 64 columns at a time; one exponent per column of the block
    const int b = local - pr.mt * pr.kt;
    const int nt = b / pr.kt, kb = b % pr.kt;
    const int64_t base = pr.b_row0 + (int64_t)b * kPackBN;
    const bool vec = al16(pr.B) && (pr.p & 3) == 0;
    for (int c0 = 0; c0 < kPackBN; c0 += 64) {
      float4 vs[8];
#pragma unroll
      for (int it = 0; it < 8; it++) {
        const int q = tid + it * 256;  // 128 k rows x 16 vectors of 4 columns
        const int kk = q / 16, c4 = q % 16;
        const int64_t k = (int64_t)kb * kBK + kk;
        const int64_t j = (int64_t)nt * kPackBN + c0 + 4 * c4;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (k < pr.m) {
          const float *src = pr.B + k * pr.p + j;
          if (vec && j + 4 <= pr.p) {
            v = __ldcs(reinterpret_cast<const float4 *>(src));
          } else {
            if (j < pr.p) v.x = src[0];
            if (j + 1 < pr.p) v.y = src[1];
            if (j + 2 < pr.p) v.z = src[2];
            if (j + 3 < pr.p) v.w = src[3];
          }
        }
        vs[it] = v;
      }
#pragma unroll
      for (int it = 0; it < 8; it++) {
        const int q = tid + it * 256;
        const int kk = q / 16, c4 = q % 16;
        tile[kk][4 * c4 + 0] = vs[it].x;
        tile[kk][4 * c4 + 1] = vs[it].y;
        tile[kk][4 * c4 + 2] = vs[it].z;
        tile[kk][4 * c4 + 3] = vs[it].w;
      }
      __syncthreads();
      {
        // column maxima: four threads a column, 32 K values each
        const int c = tid & 63, q = tid >> 6;
        uint32_t mx = 0;
#pragma unroll 8
        for (int kk = 32 * q; kk < 32 * q + 32; kk++) mx = max(mx, absb(tile[kk][c]));
        colmax[q][c] = mx;
      }
      __syncthreads();
      if (tid < 64) {
        const uint32_t mx = max(max(colmax[0][tid], colmax[1][tid]), max(colmax[2][tid], colmax[3][tid]));
        const int e = pick_exponent(mx, pr.tB[(int64_t)nt * kPackBN + c0 + tid]);
        colexp[tid] = e;
        fac_b(pr)[(int64_t)kb * pr.nt * kPackBN + (int64_t)nt * kPackBN + c0 + tid] = pow2f(e);
      }
      __syncthreads();
      for (int q = tid; q < 64 * (kBK / 16); q += 256) {
        const int c = q % 64, k16 = q / 64;
        const int e = colexp[c];
        uint4 w;
        uint32_t *wp = reinterpret_cast<uint32_t *>(&w);
#pragma unroll
        for (int t = 0; t < 4; t++) {
          const int r = 16 * k16 + 4 * t;
          wp[t] = to_e4m3x4(make_float4(tile[r][c], tile[r + 1][c], tile[r + 2][c], tile[r + 3][c]),
                            e);
        }
        *reinterpret_cast<uint4 *>(pack + (base + c0 + c) * kQuads + 4 * k16) = w;
      }
      __syncthreads();
    }
  }
}


// Tiles whose exponents do not change along K.  For row tile mt of A (items
// [0, mt) of a problem) or column tile nt of B (items [mt, mt + nt)), flag 1
// when every row (column) of the tile has the same exponent in all its K
// blocks.  A product tile whose row tile and column tile are both flagged
// takes the uniform form of the tensor-core kernel: all its K blocks are
// accumulated in tensor memory and the factor 2^(e_i + e_j), the same for
// every block, is applied once; elsewhere each block is unscaled on its own.
// flags: the problem's `cnt` array, mt + nt words; item prefix `ver_start`.
__global__ void __launch_bounds__(128)
fp8blk_flag_kernel(const SplitProb *__restrict__ probs, int nprobs) {
  const int item = blockIdx.x;
  const int g =
      find_problem(probs, nprobs, nullptr, item, [](const SplitProb &q) { return q.ver_start; });
  const SplitProb &pr = probs[g];
  const int local = item - pr.ver_start;
  const bool is_a = local < pr.mt;
  const int tile = is_a ? local : local - pr.mt;
  const int64_t width = (int64_t)(is_a ? pr.mt : pr.nt) * 128;  // padded rows per K block
  const float *f = (is_a ? fac_a(pr) : fac_b(pr)) + (int64_t)tile * 128 + threadIdx.x;
  const float f0 = f[0];
  // a row (column) with a NaN or an infinity keeps its blocks' own factors
  const uint32_t whole = (is_a ? pr.sA : pr.tB)[(int64_t)tile * 128 + threadIdx.x];
  bool same = __uint_as_float(whole) <= 3.402823466e38f;
  for (int kb = 1; kb < pr.kt; kb++) same &= f[(int64_t)kb * width] == f0;
  same = __syncthreads_and(same);
  if (threadIdx.x == 0) pr.cnt[local] = same ? 1 : 0;
}

__device__ __forceinline__ bool tile_uniform(const SplitProb &pr, int mt, int nt) {
  return pr.cnt[mt] != 0 && pr.cnt[pr.mt + nt] != 0;
}

// The 128 x 256 tile that holds sub-tile (mt, nt) is uniform: the tensor-core
// kernel of tc_gemm.cu computes it (one factor per row and column), so this
// kernel skips it in every role.
__device__ __forceinline__ bool pair_uniform(const SplitProb &pr, int mt, int nt) {
  return pr.cnt[mt] != 0 && pr.cnt[pr.mt + (nt & ~1)] != 0 && pr.cnt[pr.mt + (nt | 1)] != 0;
}

// Tile t of problem g in bands of group_m row tiles (as the split path).
__device__ __forceinline__ void blk_unit(const SplitProb *__restrict__ probs, int nprobs,
                                         const int *__restrict__ map, int u, int &g, int &mt,
                                         int &nt) {
  g = find_problem(probs, nprobs, map, u, [](const SplitProb &q) { return q.unit_start; });
  const SplitProb &pr = probs[g];
  const int t = u - pr.unit_start;
  const int gm = pr.group_m;
  const int band = gm * pr.nt;
  const int first = (t / band) * gm;
  const int rows = min(pr.mt - first, gm);
  const int in = t % band;
  mt = first + in % rows;
  nt = in / rows;
}

__global__ void __launch_bounds__(kThreads, 1)
fp8blk_gemm_kernel(const __grid_constant__ CUtensorMap tmap, const SplitProb *__restrict__ probs,
                   int nprobs, const int *__restrict__ unit_map, int total_units, int *err) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t sbase = (raw + 1023u) & ~1023u;
  uint8_t *smem = smem_raw + (sbase - raw);
  const uint32_t bars = sbase + Lay::kBarOff;
  auto full_bar = [&](int s) { return bars + 8u * s; };
  auto empty_bar = [&](int s) { return bars + 8u * (kStages + s); };
  auto efull_bar = [&](int s) { return bars + 8u * (2 * kStages + s); };
  auto eempty_bar = [&](int s) { return bars + 8u * (2 * kStages + kEStages + s); };
  auto accf_bar = [&](int a) { return bars + 8u * (2 * kStages + 2 * kEStages + a); };
  auto acce_bar = [&](int a) { return bars + 8u * (2 * kStages + 2 * kEStages + kAccs + a); };
  const uint32_t drain_bar = bars + 8u * (2 * kStages + 2 * kEStages + 2 * kAccs);
  uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(smem + Lay::kMiscOff);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_holder), 512);
    tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; s++) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int s = 0; s < kEStages; s++) {
      mbar_init(efull_bar(s), 1);
      mbar_init(eempty_bar(s), kWorkers / 32);  // one arrival per worker warp
    }
    for (int a = 0; a < kAccs; a++) {
      mbar_init(accf_bar(a), 1);
      mbar_init(acce_bar(a), kWorkers / 32);
    }
    mbar_init(drain_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *reinterpret_cast<volatile uint32_t *>(tmem_holder);

  if (warp == 0) {
    if (lane == 0) {
      // ---------------------------------------------------- TMA producer
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap)) : "memory");
      int stage = 0, es = 0;
      uint32_t phase = 0, ephase = 0, issued = 0, eissued = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < total_units && ok; u += gridDim.x) {
        int g, mt, nt;
        blk_unit(probs, nprobs, unit_map, u, g, mt, nt);
        const SplitProb &pr = probs[g];
        if (pair_uniform(pr, mt, nt)) continue;
        const int64_t abase = pr.a_row0 + (int64_t)mt * pr.kt * kTcBM;
        // sub-tile nt of 128 columns: half nt & 1 of pack tile nt >> 1
        const int64_t bbase = pr.b_row0 + (int64_t)(nt >> 1) * pr.kt * kPackBN + (nt & 1) * kBN;
        const bool uni = tile_uniform(pr, mt, nt);
        for (int kb = 0; kb < pr.kt; kb++) {
          if (!mbar_wait(empty_bar(stage), phase ^ 1u, err, 21, true, kWaitNs)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(full_bar(stage), (uint32_t)Lay::kStage);
          ++issued;
          const uint32_t st = sbase + (uint32_t)(stage * Lay::kStage);
          tma_load_2d(st, &tmap, 0, (int)(abase + (int64_t)kb * kTcBM), full_bar(stage));
          tma_load_2d(st + Lay::kA, &tmap, 0, (int)(bbase + (int64_t)kb * kPackBN), full_bar(stage));
          if (++stage == kStages) {
            stage = 0;
            phase ^= 1u;
          }
          // the block's row and column factors (a uniform tile: block 0's only)
          if (uni && kb > 0) continue;
          if (!mbar_wait(eempty_bar(es), ephase ^ 1u, err, 21, true, kWaitNs)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(efull_bar(es), (uint32_t)Lay::kESlot);
          ++eissued;
          const uint32_t ed = sbase + (uint32_t)(Lay::kEOff + es * Lay::kESlot);
          bulk_load(ed, fac_a(pr) + ((int64_t)kb * pr.mt + mt) * kTcBM, 512, efull_bar(es));
          bulk_load(ed + 512, fac_b(pr) + ((int64_t)kb * pr.nt + nt) * kBN, 512, efull_bar(es));
          if (++es == kEStages) {
            es = 0;
            ephase ^= 1u;
          }
        }
      }
      if (!ok) {
        // copies in flight must land before the shared memory goes away
        for (uint32_t j = issued > kStages ? issued - kStages : 0; j < issued; j++)
          mbar_wait(full_bar((int)(j % kStages)), (j / kStages) & 1u, err, 21, false, kDrainNs);
        for (uint32_t j = eissued > kEStages ? eissued - kEStages : 0; j < eissued; j++)
          mbar_wait(efull_bar((int)(j % kEStages)), (j / kEStages) & 1u, err, 21, false, kDrainNs);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------------------------------------------- MMA issuer
      const uint32_t idesc = make_idesc<kTcE4m3>(kBN);
      int stage = 0, acc = 0;
      uint32_t phase = 0, aphase = 0;
      bool ok = true, any = false;
      for (int u = blockIdx.x; u < total_units && ok; u += gridDim.x) {
        int g, mt, nt;
        blk_unit(probs, nprobs, unit_map, u, g, mt, nt);
        if (pair_uniform(probs[g], mt, nt)) continue;
        const int kt = probs[g].kt;
        // a uniform tile accumulates all its K blocks in one accumulator;
        // otherwise each block takes an accumulator of its own
        const bool uni = tile_uniform(probs[g], mt, nt);
        for (int kb = 0; kb < kt; kb++) {
          const bool fresh = !uni || kb == 0;  // the block starts an accumulator
          if ((fresh && !mbar_wait(acce_bar(acc), aphase ^ 1u, err, 22, true, kWaitNs)) ||
              !mbar_wait(full_bar(stage), phase, err, 22, true, kWaitNs)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t st = sbase + (uint32_t)(stage * Lay::kStage);
          const uint64_t a0 = kmajor_desc<128>(st), b0 = kmajor_desc<128>(st + Lay::kA);
          const uint32_t d_tmem = tmem_base + (uint32_t)(acc * kBN);
#pragma unroll
          for (int kk = 0; kk < kBK / 32; kk++) {  // 32 e4m3 = 32 bytes per MMA
            const uint64_t adv = (uint64_t)(kk * 32) >> 4;
            tc_mma_f8(d_tmem, a0 + adv, b0 + adv, idesc, (kk != 0 || !fresh) ? 1u : 0u);
          }
          any = true;
          tc_commit(empty_bar(stage));
          if (++stage == kStages) {
            stage = 0;
            phase ^= 1u;
          }
          if (!uni || kb == kt - 1) {  // the accumulator is complete
            tc_commit(accf_bar(acc));
            if (++acc == kAccs) {
              acc = 0;
              aphase ^= 1u;
            }
          }
        }
      }
      if (!ok && any) {
        tc_commit(drain_bar);
        mbar_wait(drain_bar, 0, err, 22, false, kDrainNs);
      }
    }
  } else {
    // ---------------------------------------------------------- workers
    // warps 2..9: TMEM lane quarter warp % 4, column half (warp - 2) / 4
    const int wq = warp & 3, ch = (warp - 2) >> 2;
    const int row = wq * 32 + lane;
    const uint32_t tlane = (uint32_t)(wq * 32) << 16;
    int acc = 0, es = 0;
    uint32_t aphase = 0, ephase = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < total_units && ok; u += gridDim.x) {
      int g, mt, nt;
      blk_unit(probs, nprobs, unit_map, u, g, mt, nt);
      const SplitProb &pr = probs[g];
      if (pair_uniform(pr, mt, nt)) continue;
      // column pairs, packed for the paired FP32 instructions
      uint64_t sum[kWCols / 2];
#pragma unroll
      for (int c = 0; c < kWCols / 2; c++) sum[c] = 0ull;
      // a uniform tile's accumulator holds all its K blocks (one factor slot)
      const int nacc = tile_uniform(pr, mt, nt) ? 1 : pr.kt;
      for (int kb = 0; kb < nacc; kb++) {
        bool w = mbar_wait(efull_bar(es), ephase, err, 23, true, kWaitNs) &&
                 mbar_wait(accf_bar(acc), aphase, err, 23, true, kWaitNs);
        // agreement within the warp (tcgen05.ld is warp-collective); warps
        // that give up leave on their own, the others then run out of time too
        if (!__all_sync(0xffffffffu, w)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const float *fx = reinterpret_cast<const float *>(smem + Lay::kEOff + es * Lay::kESlot);
        const float fr = fx[row];
        const uint64_t fr2 = pack_f32x2(__float_as_uint(fr), __float_as_uint(fr));
        // this warp's columns' factors, two per 8-byte word
        const uint64_t *fc2 = reinterpret_cast<const uint64_t *>(fx + 128 + ch * kWCols);
        uint32_t v[kWCols];
        const uint32_t ta = tmem_base + tlane + (uint32_t)(acc * kBN + ch * kWCols);
#pragma unroll
        for (int c0 = 0; c0 < kWCols; c0 += 16)
          tmem_ld_32x32b_x16(ta + c0, *reinterpret_cast<uint32_t(*)[16]>(&v[c0]));
        tmem_ld_wait();
        // v 2^(e_j) 2^(e_i): both factors are powers of two, so each product
        // is exact and one rounding (the addition) remains; two columns per
        // instruction (mul.rn / fma.rn on FP32 pairs: each half rounds as the
        // scalar instruction would)
#pragma unroll
        for (int c = 0; c < kWCols / 2; c++)
          sum[c] = fma_f32x2(mul_f32x2(pack_f32x2(v[2 * c], v[2 * c + 1]), fc2[c]), fr2, sum[c]);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(acce_bar(acc));
          mbar_arrive(eempty_bar(es));
        }
        if (++acc == kAccs) {
          acc = 0;
          aphase ^= 1u;
        }
        if (++es == kEStages) {
          es = 0;
          ephase ^= 1u;
        }
      }
      if (!ok) break;
      // the tile's rows: kWCols consecutive columns of one row per thread
      const int64_t i = (int64_t)mt * kTcBM + row;
      const int64_t j0 = (int64_t)nt * kBN + ch * kWCols;
      if (i < pr.n) {
        float out[kWCols];
#pragma unroll
        for (int c = 0; c < kWCols / 2; c++) unpack_f32x2(sum[c], out[2 * c], out[2 * c + 1]);
        float *dst = pr.C + i * pr.p + j0;
        if (al16(pr.C) && (pr.p & 3) == 0 && j0 + kWCols <= pr.p) {
#pragma unroll
          for (int c = 0; c < kWCols; c += 4)
            __stcs(reinterpret_cast<float4 *>(dst + c),
                   make_float4(out[c], out[c + 1], out[c + 2], out[c + 3]));
        } else {
#pragma unroll
          for (int c = 0; c < kWCols; c++)
            if (j0 + c < pr.p) __stcs(dst + c, out[c]);
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem_base, 512);
  }
}

// ---------------------------------------------------------------- host side
PFN_cuTensorMapEncodeTiled_v12000 blk_encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// the pack region as rows of 128 bytes, boxes of 128 rows, 128-byte swizzle
cudaError_t blk_pack_map(CUtensorMap *map, void *base, int64_t rows) {
  auto enc = blk_encode_fn();
  if (!enc) return cudaErrorNotSupported;
  cuuint64_t dims[2] = {(cuuint64_t)kPackRowBytes, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kPackRowBytes};
  cuuint32_t box[2] = {128u, 128u};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, base, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

namespace {

mm_status fp8_blocks_launch(Scratch &ws, std::vector<SplitProb> &blk, std::vector<SplitProb> &tc,
                            int64_t rows, int64_t exps, int64_t maxw, int64_t blk_units,
                            int64_t tc_units, int64_t packs, int64_t flag_items,
                            int64_t max_items_all, cudaStream_t s) {
  if (rows > 0x7fffffffLL || blk_units > 0x7fffffffLL || packs > 0x7fffffffLL ||
      flag_items > 0x7fffffffLL)
    return MM_EINVAL;
  const int np = (int)blk.size();
  // layout: packs | factors (FP32) | maxima words | tile flags | both tables
  // (one copy) | unit maps and the pack map
  const size_t pack_bytes = (size_t)rows * kPackRowBytes;
  const size_t exp_off = (pack_bytes + 255) & ~(size_t)255;
  const size_t max_off = (exp_off + (size_t)exps * 4 + 255) & ~(size_t)255;
  const size_t flag_off = (max_off + (size_t)maxw * 4 + 255) & ~(size_t)255;
  const size_t tab_off = (flag_off + (size_t)flag_items * 4 + 255) & ~(size_t)255;
  const size_t tab_bytes = (size_t)np * sizeof(SplitProb);
  // tensor maps over the C matrices for the tensor-core kernel's tiled
  // stores (tables of up to kMaxCMaps products), after the two tables
  constexpr size_t kMaxCMaps = 8192, kMapBytes = 128;
  const size_t cmap_rel = (2 * tab_bytes + 63) & ~(size_t)63;
  const size_t cmap_bytes = (size_t)np <= kMaxCMaps ? (size_t)np * kMapBytes : 0;
  const size_t map_off = (tab_off + cmap_rel + cmap_bytes + 255) & ~(size_t)255;
  const size_t map_ints = np > 1 ? (size_t)(blk_units + tc_units + packs) : 0;
  cudaError_t e = ws.reserve(map_off + map_ints * sizeof(int), s);
  if (e != cudaSuccess) return note_cuda(e);
  uint8_t *base = static_cast<uint8_t *>(ws.ptr);
  for (int g = 0; g < np; g++) {
    for (SplitProb *sp : {&blk[(size_t)g], &tc[(size_t)g]}) {
      sp->pA = reinterpret_cast<uint32_t *>(base + exp_off) + (uintptr_t)sp->pA;
      sp->pB = reinterpret_cast<uint32_t *>(base + exp_off) + (uintptr_t)sp->pB;
      sp->sA = reinterpret_cast<uint32_t *>(base + max_off) + (uintptr_t)sp->sA;
      sp->tB = reinterpret_cast<uint32_t *>(base + max_off) + (uintptr_t)sp->tB;
    }
    blk[(size_t)g].cnt = reinterpret_cast<int *>(base + flag_off) + (uintptr_t)blk[(size_t)g].cnt;
    tc[(size_t)g].cnt = blk[(size_t)g].cnt;  // the tensor-core kernel reads the same flags
  }
  SplitProb *d_blk = reinterpret_cast<SplitProb *>(base + tab_off);
  SplitProb *d_tc = d_blk + np;
  const void *d_cmaps = cmap_bytes ? static_cast<const void *>(base + tab_off + cmap_rel) : nullptr;
  {
    std::vector<uint8_t> blob(cmap_rel + cmap_bytes, 0);
    for (size_t g = 0; cmap_bytes && g < (size_t)np; g++) {
      SplitProb &t = tc[g];
      if (tc_c_map_ok(t.C, t.n, t.p) &&
          encode_c_map(blob.data() + cmap_rel + g * kMapBytes, t.C, t.n, t.p) == cudaSuccess)
        t.c_tma = (int32_t)g + 1;
    }
    std::memcpy(blob.data(), blk.data(), tab_bytes);
    std::memcpy(blob.data() + tab_bytes, tc.data(), tab_bytes);
    e = ws.stage.copy_to_device(d_blk, blob.data(), blob.size(), s);
  }
  // whole-row and whole-column maxima first (zeroed: columns merge by atomicMax)
  if (e == cudaSuccess) e = cudaMemsetAsync(base + max_off, 0, (size_t)maxw * 4, s);
  if (e != cudaSuccess) return note_cuda(e);
  {
    TraceScope ts("fp8_max", s);
    fp8blk_max_kernel<<<(unsigned)max_items_all, 256, 0, s>>>(d_blk, np);
    if ((e = cudaGetLastError()) != cudaSuccess) return note_cuda(e);
  }
  int *blk_map = nullptr, *tc_map = nullptr, *pack_map = nullptr;
  if (np > 1) {
    blk_map = reinterpret_cast<int *>(base + map_off);
    tc_map = blk_map + blk_units;
    pack_map = tc_map + tc_units;
    e = launch_split_maps(d_blk, np, blk_map, nullptr, nullptr, s);
    if (e == cudaSuccess) e = launch_split_maps(d_tc, np, tc_map, pack_map, nullptr, s);
    if (e != cudaSuccess) return note_cuda(e);
  }
  {
    TraceScope ts("fp8_pack", s);
    fp8blk_pack_kernel<<<(unsigned)packs, 256, 0, s>>>(d_tc, np, pack_map,
                                                       static_cast<uint32_t *>(ws.ptr));
    if ((e = cudaGetLastError()) != cudaSuccess) return note_cuda(e);
    fp8blk_flag_kernel<<<(unsigned)flag_items, 128, 0, s>>>(d_blk, np);
    if ((e = cudaGetLastError()) != cudaSuccess) return note_cuda(e);
  }
  // the uniform 128 x 256 tiles: one factor per row and column
  TcConfig cfg{128, 4, 0};
  cfg.max_bn = kPackBN;
  e = launch_tc(kTcE4m3, d_tc, np, (int)tc_units, tc_map, nullptr, ws.ptr, rows, cfg, g_ctx.d_err,
                s, nullptr, 1, d_cmaps);
  if (e != cudaSuccess) return note_cuda(e);
  // the other tiles, K block by K block
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [] {
    attr_err = cudaFuncSetAttribute(fp8blk_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    Lay::kSmem);
  });
  if (attr_err != cudaSuccess) return note_cuda(attr_err);
  CUtensorMap map;
  if ((e = blk_pack_map(&map, ws.ptr, rows)) != cudaSuccess) return note_cuda(e);
  const int grid = (int)std::min<int64_t>(blk_units, sm_count());
  TraceScope ts("fp8_blk", s);
  fp8blk_gemm_kernel<<<grid, kThreads, Lay::kSmem, s>>>(map, d_blk, np, blk_map, (int)blk_units,
                                                        g_ctx.d_err);
  return note_cuda(cudaGetLastError());
}

}  // namespace

size_t fp8_blocks_scratch_bytes(int64_t n, int64_t m, int64_t p) {
  if (n <= 0 || m <= 0 || p <= 0) return 0;
  const int64_t mt = ceil_div(n, kTcBM), nt = ceil_div(p, kPackBN), kt = ceil_div(m, kBK);
  // packs and factors, maxima, tile flags, two tables, unit maps
  return (size_t)(mt * kTcBM + nt * kPackBN) * kt * (kPackRowBytes + 4) +
         (size_t)(mt * kTcBM + nt * kPackBN) * 4 + (size_t)(mt + 2 * nt) * 4 +
         2 * sizeof(SplitProb) + 256 + (size_t)mt * nt * 12 + 4096;
}

// Two tables over the same packs: `blk` for the blockwise kernel (N sub-tiles
// of 128 columns: nt = 2 x the pack tiles of B) and `tc` for the tensor-core
// kernel of split_prep/tc_gemm (128 x 256 tiles, one factor per row and
// column from the maxima words).  The pack kernel runs over `tc`.
mm_status run_fp8_blocks(Scratch &ws, const mm_problem *probs, int count, cudaStream_t s) {
  std::vector<SplitProb> blk, tc;
  int64_t rows = 0, exps = 0, maxw = 0, blk_units = 0, tc_units = 0, packs = 0, flag_items = 0,
          max_items_all = 0;
  for (int g = 0; g < count; g++) {
    const mm_problem &q = probs[g];
    if (q.n == 0 || q.p == 0) continue;
    if (q.m == 0) {
      cudaError_t e = cudaMemsetAsync(q.C, 0, (size_t)(q.n * q.p) * sizeof(float), s);
      if (e != cudaSuccess) return note_cuda(e);
      continue;
    }
    SplitProb sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.A = static_cast<const float *>(q.A);
    sp.B = static_cast<const float *>(q.B);
    sp.C = static_cast<float *>(q.C);
    sp.n = (int32_t)q.n;
    sp.m = (int32_t)q.m;
    sp.p = (int32_t)q.p;
    sp.group_m = 16;
    sp.mt = (int32_t)ceil_div(q.n, kTcBM);
    const int32_t ntp = (int32_t)ceil_div(q.p, kPackBN);  // pack tiles of B
    sp.kt = (int32_t)ceil_div(q.m, kBK);
    sp.a_row0 = rows;
    rows += (int64_t)sp.mt * sp.kt * kTcBM;
    sp.b_row0 = rows;
    rows += (int64_t)ntp * sp.kt * kPackBN;
    sp.pA = reinterpret_cast<uint32_t *>((uintptr_t)exps);  // offsets, fixed below
    exps += (int64_t)sp.kt * sp.mt * kTcBM;
    sp.pB = reinterpret_cast<uint32_t *>((uintptr_t)exps);
    exps += (int64_t)sp.kt * ntp * kPackBN;
    sp.sA = reinterpret_cast<uint32_t *>((uintptr_t)maxw);
    maxw += (int64_t)sp.mt * kTcBM;
    sp.tB = reinterpret_cast<uint32_t *>((uintptr_t)maxw);
    maxw += (int64_t)ntp * kPackBN;
    sp.pack_start = (int32_t)packs;
    packs += (int64_t)sp.mt * sp.kt + (int64_t)ntp * sp.kt;
    SplitProb b = sp, t = sp;
    b.bn = kBN;
    b.nt = 2 * ntp;
    b.unit_start = (int32_t)blk_units;
    blk_units += (int64_t)b.mt * b.nt;
    b.ver_start = (int32_t)flag_items;  // uniform-exponent flags of its tiles
    b.cnt = reinterpret_cast<int *>((uintptr_t)flag_items);  // offset, fixed below
    flag_items += (int64_t)b.mt + b.nt;
    b.split_s = 1;
    b.split_from = (int32_t)max_items_all;  // prefix of its maxima items
    max_items_all += max_items(q.n, q.m, q.p);
    t.bn = kPackBN;
    t.nt = ntp;
    t.unit_start = (int32_t)tc_units;
    tc_units += (int64_t)t.mt * t.nt;
    t.split_from = t.mt * t.nt;
    t.split_s = 1;
    blk.push_back(b);
    tc.push_back(t);
  }
  if (blk.empty()) return MM_OK;
  if (max_items_all > 0x7fffffffLL) return MM_EINVAL;
  return fp8_blocks_launch(ws, blk, tc, rows, exps, maxw, blk_units, tc_units, packs, flag_items,
                           max_items_all, s);
}

}  // namespace mm
