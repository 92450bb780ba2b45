// Fused split-K tensor-core product for under-filled FP32 products.
//
// A product with few 128 x 128 output tiles (or a long inner dimension) leaves
// most of the 152 SMs idle on the packed path (split_prep.cu + tc_gemm.cu),
// and its four dependent launches cost more than its arithmetic.  This kernel
// computes such a product in ONE launch:
//
//   * Work units are (output tile, K slice): the inner dimension of each tile
//     is cut into S slices (S = Q * CS), one CTA per slice, CS CTAs of the
//     same tile forming one thread-block cluster.
//   * TMA copies the FP32 operands straight from the caller's matrices (no
//     pack pass) into two shared-memory staging buffers, one K block of 64 at
//     a time (zero fill past the edges); eight worker warps split each block
//     into bf16 parts (x3: hi, lo; x6: hi, mid, lo - the split of Henry, Tang
//     & Heinecke, ARITH 2019) and write them into shared memory in the
//     128-byte-swizzled K-major layout that tcgen05 reads (B transposed on
//     the way).
//   * One thread issues the tcgen05 MMAs of the block (hi.hi + hi.lo + lo.hi,
//     or the six products of the three-part split) into one of two tensor-
//     memory accumulators; the same worker warps load the block's FP32
//     partial product (tcgen05.ld) and add it into registers, so every block of 64
//     terms is accumulated on the tensor cores and the blocks are summed with
//     round-to-nearest FP32 additions.
//   * Scaling: a block whose non-zero entries all lie in [2^-40, 2^40] is
//     split as it is (power-of-two scaling would give the same bits there);
//     a block holding anything outside that range (or a NaN / infinity) is
//     split after scaling each row of A and each column of B by the power of
//     two of its largest magnitude within the block, and its partial product
//     is unscaled exactly by 2^(s_i + t_j) before it is added.  The choice is
//     made per block from the block's own entries, so it is deterministic.
//   * Reduction of the S slice partials of a tile, in a fixed order: the CS
//     CTAs of a cluster exchange their partials through distributed shared
//     memory, CTA r adding rank 0..CS-1 for its own eighth (CS-th) of the
//     tile's rows; with Q > 1 clusters per tile, each writes its summed rows
//     to a global slot and counts itself on that row chunk's counter, and the
//     cluster that arrives last adds the Q slots in order 0..Q-1.  No CTA
//     waits for a CTA outside its cluster, and the sum does not depend on
//     which cluster finishes last.
//
// The product computed is the paper's Cauchy product (Section "Implementacje
// algorytmow"); the split-K decomposition, the split precision and the
// cluster reduction are this library's design for GB300.  Every mbarrier wait
// is bounded; a wait that runs out sets the device error flag, the CTA skips
// its remaining work but still takes part in its cluster's barriers, and the
// reduction then leaves C untouched (the call reports MM_ETIMEOUT).
#include <cooperative_groups.h>
#include <cudaTypedefs.h>

#include "ctx.h"
#include "tc_ptx.cuh"

namespace mm {
namespace {

using namespace tcx;

constexpr int kFBN = 128;                 // N tile
constexpr int kFBK = 64;                  // K block: one 128-byte row of bf16
constexpr int kFWorkers = 256;            // warps 0-7: conversion and accumulation
constexpr int kFThreads = kFWorkers + 32; // warp 8: tensor memory and the MMAs
constexpr int kFMma = 8;
constexpr uint32_t kFTmemCols = 256;      // two 128-column FP32 accumulators
constexpr uint64_t kFWaitNs = 4000000000ull;
constexpr uint64_t kFDrainNs = 200000000ull;
constexpr int kFRedPitch = kFBN + 1;      // floats per row of the reduction buffer

// Shared-memory layout for PARTS bf16 parts per operand: two FP32 staging
// buffers that TMA fills (A block 128 x 64, then B block 64 x 128), one bf16
// operand buffer (A parts, then B parts, 128 rows of 128 bytes each, 128-byte
// swizzle), two scale slots (one per tensor-memory accumulator), barriers.
template <int PARTS>
struct FusedLayout {
  static constexpr int kStgA = kTcBM * kFBK * 4;              // 32 KB
  static constexpr int kStgB = kFBK * kFBN * 4;               // 32 KB
  static constexpr int kStgBytes = kStgA + kStgB;
  static constexpr int kPartBytes = 128 * 128;                // 128 rows x 128 bytes
  static constexpr int kOpndOff = 2 * kStgBytes;
  static constexpr int kOpndBytes = 2 * PARTS * kPartBytes;   // A parts, then B parts
  static constexpr int kScaleOff = kOpndOff + kOpndBytes;     // per accumulator slot:
  static constexpr int kScaleSlot = 128 * 2 + 128 * 2 + 16;   //   sa[128], sb[128] (int16), flags
  static constexpr int kBarOff = kScaleOff + 2 * kScaleSlot;
  // stage_full[2], opnd_full, opnd_empty, acc_full[2], drain
  static constexpr int kNumBars = 7;
  static constexpr int kMiscOff = kBarOff + kNumBars * 8;     // tmem holder, last flag
  static constexpr int kSmemBytes = kMiscOff + 64 + 1024;     // + alignment slack
  static_assert(128 * kFRedPitch * 4 <= kOpndOff, "reduction buffer fits the staging");
  static_assert(kFWorkers / 32 * 128 * 4 <= kStgA, "column maxima fit the A staging");
};

__device__ __forceinline__ uint32_t abs_bits(float x) { return __float_as_uint(x) & 0x7fffffffu; }

// An entry the unscaled split handles exactly like the scaled one: zero, or a
// magnitude in [2^-40, 2^40] (NaN and infinity fall outside).
__device__ __forceinline__ bool in_range(float x) {
  const uint32_t b = abs_bits(x);
  return b == 0u || (b >= 0x2B800000u && b <= 0x53800000u);
}

__device__ __forceinline__ bool in_range4(float4 v) {
  return in_range(v.x) && in_range(v.y) && in_range(v.z) && in_range(v.w);
}

__device__ __forceinline__ uint32_t max4_bits(float4 v) {
  const uint32_t a = max(abs_bits(v.x), abs_bits(v.y)), b = max(abs_bits(v.z), abs_bits(v.w));
  return max(a, b);
}

// Splits four values, scaled by 2^-s when SCALED, into PARTS groups of four
// bf16 (8 bytes each): part 0 = RN(y), part q = RN(y - parts 0..q-1); every
// remainder is exact in FP32.
template <int PARTS>
__device__ __forceinline__ void split4f(float4 x, bool scaled, int s, uint2 (&out)[PARTS]) {
  float y[4] = {x.x, x.y, x.z, x.w};
  if (scaled) {
#pragma unroll
    for (int e = 0; e < 4; e++) y[e] = scale_pow2(y[e], -s);
  }
#pragma unroll
  for (int q = 0; q < PARTS; q++) {
    const __nv_bfloat162 a = __floats2bfloat162_rn(y[0], y[1]);
    const __nv_bfloat162 b = __floats2bfloat162_rn(y[2], y[3]);
    const float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
    y[0] -= fa.x;
    y[1] -= fa.y;
    y[2] -= fb.x;
    y[3] -= fb.y;
    out[q] = make_uint2(*reinterpret_cast<const uint32_t *>(&a),
                        *reinterpret_cast<const uint32_t *>(&b));
  }
}

// Byte offset of the 8-byte group kq (four bf16, 0..15) of row r in a K-major
// operand part of 128-byte rows, with the 128-byte swizzle TMA would apply:
// the 16-byte chunk c of row r sits at chunk c ^ (r mod 8).
__device__ __forceinline__ uint32_t swz(int r, int kq) {
  return (uint32_t)(r * 128 + ((((kq >> 1) ^ (r & 7)) << 4) | ((kq & 1) << 3)));
}

// AND of a predicate over the worker threads (named barrier 1), and a plain
// barrier among them (named barrier 2).
__device__ __forceinline__ bool work_all(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.and.pred p, 1, %2, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(kFWorkers)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ void work_sync() {
  asm volatile("bar.sync 2, %0;" ::"n"(kFWorkers) : "memory");
}

__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release;\n\t"
               "barrier.cluster.wait.acquire;" ::: "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}



template <int PARTS>
__global__ void __launch_bounds__(kFThreads, 1)
tc_fused_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                const __grid_constant__ FusedProb pr, int *err) {
  using L = FusedLayout<PARTS>;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t sbase = (raw + 1023u) & ~1023u;
  uint8_t *smem = smem_raw + (sbase - raw);
  const uint32_t bars = sbase + L::kBarOff;
  auto stage_full = [&](int b) { return bars + 8u * b; };
  const uint32_t opnd_full = bars + 16u, opnd_empty = bars + 24u;
  auto acc_full = [&](int a) { return bars + 8u * (4 + a); };
  const uint32_t drain_bar = bars + 48u;
  uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(smem + L::kMiscOff);
  volatile int *last_flag = reinterpret_cast<volatile int *>(smem + L::kMiscOff + 16);
  auto slot = [&](int a) { return reinterpret_cast<int16_t *>(smem + L::kScaleOff + a * L::kScaleSlot); };

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile = (int)blockIdx.x / pr.S, h = (int)blockIdx.x % pr.S;
  const int cs = pr.S / pr.Q;
  const int q = h / cs;
  const int crank = cs > 1 ? (int)cluster_rank() : 0;  // == h % cs
  const int mt_i = tile / pr.nt, nt_i = tile % pr.nt;
  const int64_t row0 = (int64_t)mt_i * kTcBM, col0 = (int64_t)nt_i * kFBN;
  const int kb0 = (int)((int64_t)h * pr.kb / pr.S);
  const int nkb = (int)((int64_t)(h + 1) * pr.kb / pr.S) - kb0;

  if (warp == kFMma) {
    tmem_alloc(smem_u32(tmem_holder), kFTmemCols);
    tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; i++) {
      mbar_init(stage_full(i), 1);
      mbar_init(acc_full(i), 1);
    }
    mbar_init(opnd_full, kFWorkers);
    mbar_init(opnd_empty, 1);
    mbar_init(drain_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *reinterpret_cast<volatile uint32_t *>(tmem_holder);
  // launched as a programmatic dependent of the stream's previous kernel:
  // the set-up above may overlap its end; nothing in global memory is read
  // or written before it has finished
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

  if (warp < kFMma) {
    // ------------------------------------------------------------ workers
    // convert block j, then (while the MMAs of block j run) add the partial
    // product of block j - 1 into this thread's 64 accumulator columns
    const int wt = threadIdx.x;  // 0..255
    const int kq = wt & 15;
    const int rows_in = (int)min((int64_t)kTcBM, (int64_t)pr.n - row0);
    const int wq = warp & 3, ch = warp >> 2;  // TMEM lane quarter, column half
    const int row = wq * 32 + lane;           // row of the tile this thread accumulates
    const uint32_t tlane = (uint32_t)(wq * 32) << 16;
    float acc[kFBN / 2];
#pragma unroll
    for (int c = 0; c < kFBN / 2; c++) acc[c] = 0.0f;
    // TMA: block j's A box (64 K x 128 rows) and B box (128 columns x 64 K)
    // into staging buffer j % 2; parts outside A or B read as zero
    auto issue_stage = [&](int j) {
      const int b = j & 1;
      const uint32_t dst = sbase + (uint32_t)(b * L::kStgBytes);
      const int kx = (kb0 + j) * kFBK;
      mbar_arrive_expect_tx(stage_full(b), (uint32_t)L::kStgBytes);
      tma_load_2d(dst, &map_a, kx, (int)row0, stage_full(b));
      tma_load_2d(dst + L::kStgA, &map_b, (int)col0, kx, stage_full(b));
    };
    // adds block jb's partial product (accumulator jb % 2) into acc
    auto accumulate = [&](int jb) -> bool {
      const int a = jb & 1;
      const bool ok = mbar_wait(acc_full(a), (uint32_t)((jb >> 1) & 1), err, 13, true, kFWaitNs);
      __syncwarp();
      if (!work_all(ok)) return false;
      tc_fence_after();
      const int16_t *sa = slot(a), *sb = sa + 128;
      const int *flags = reinterpret_cast<const int *>(sa + 256);
      const bool scaled = (flags[0] | flags[1]) != 0;
      const int sr = sa[row];
#pragma unroll
      for (int c0 = 0; c0 < kFBN / 2; c0 += 16) {
        uint32_t v[16];
        __syncwarp();
        tmem_ld_32x32b_x16(tmem_base + tlane + (uint32_t)(a * kFBN + ch * (kFBN / 2) + c0), v);
        tmem_ld_wait();
        if (!scaled) {
#pragma unroll
          for (int e = 0; e < 16; e++) acc[c0 + e] += __uint_as_float(v[e]);
        } else {
#pragma unroll
          for (int e = 0; e < 16; e++)
            acc[c0 + e] += scale_pow2(__uint_as_float(v[e]), sr + (int)sb[ch * (kFBN / 2) + c0 + e]);
        }
      }
      tc_fence_before();
      return true;
    };
    int issued = 0;
    if (wt == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_a)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_b)) : "memory");
      for (; issued < 2 && issued < nkb; issued++) issue_stage(issued);
    }
    int j = 0;
    bool ok = true;
    for (; j < nkb; j++) {
      const int a = j & 1, u = j >> 1;
      bool w_ok = mbar_wait(stage_full(a), (uint32_t)(u & 1), err, 11, true, kFWaitNs);
      w_ok = w_ok && (j == 0 || mbar_wait(opnd_empty, (uint32_t)((j - 1) & 1), err, 11, true, kFWaitNs));
      __syncwarp();
      // also: every worker is done reading scale slot a (block j - 2)
      if (!work_all(w_ok)) {
        ok = false;
        break;
      }
      const float *stg_a = reinterpret_cast<const float *>(smem + a * L::kStgBytes);
      const float *stg_b = stg_a + kTcBM * kFBK;
      uint8_t *op_a = smem + L::kOpndOff;
      uint8_t *op_b = op_a + PARTS * L::kPartBytes;
      int16_t *sa = slot(a), *sb = sa + 128;
      int *flags = reinterpret_cast<int *>(sa + 256);
      // A block: rows r = wt/16 + 16 it, four values at K offset 4 kq (a half
      // warp reads one row's 256 bytes).  Rows past the end of A are skipped:
      // their operand rows only feed rows of the product that are not stored
      {
        float4 x[8];
        bool good = true;
#pragma unroll
        for (int it = 0; it < 8; it++) {
          const int r = (wt >> 4) + 16 * it;
          x[it] = r < rows_in ? reinterpret_cast<const float4 *>(stg_a)[r * (kFBK / 4) + kq]
                              : make_float4(0.f, 0.f, 0.f, 0.f);
          good &= in_range4(x[it]);
        }
        __syncwarp();
        const bool scaled = !work_all(good);
#pragma unroll
        for (int it = 0; it < 8; it++) {
          const int r = (wt >> 4) + 16 * it;
          int sc = 0;
          if (scaled) {
            uint32_t mx = max4_bits(x[it]);
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            sc = scale_exponent(mx);
          }
          if (kq == 0) sa[r] = (int16_t)sc;
          if (r < rows_in) {
            uint2 part[PARTS];
            split4f<PARTS>(x[it], scaled, sc, part);
#pragma unroll
            for (int pp = 0; pp < PARTS; pp++)
              *reinterpret_cast<uint2 *>(op_a + pp * L::kPartBytes + swz(r, kq)) = part[pp];
          }
        }
        if (wt == 0) flags[0] = scaled ? 1 : 0;
      }
      // B block: warp w takes K rows 8 w .. 8 w + 7, lane l the columns
      // l + 32 c (c = 0..3): eight consecutive K values of a column, i.e. one
      // 16-byte chunk of a row of the K-major (transposed) B operand; the
      // rows a warp writes are 32 apart in c and consecutive in l, so each
      // chunk store spreads over all banks (rows 4 l + c had put 16 lanes on
      // each bank group)
      {
        const int w = warp, l = lane;
        bool col_in[4];  // columns past B: as rows past A
        float y[8][4];
        bool good = true;
#pragma unroll
        for (int c = 0; c < 4; c++) col_in[c] = col0 + l + 32 * c < pr.p;
#pragma unroll
        for (int t = 0; t < 8; t++) {
#pragma unroll
          for (int c = 0; c < 4; c++)
            y[t][c] = col_in[c] ? stg_b[(8 * w + t) * kFBN + l + 32 * c] : 0.0f;
          good &= in_range4(make_float4(y[t][0], y[t][1], y[t][2], y[t][3]));
        }
        __syncwarp();
        const bool scaled = !work_all(good);  // also: every worker is done with stg_a
        int sc[4] = {0, 0, 0, 0};
        if (scaled) {
          uint32_t mx[4] = {0, 0, 0, 0};
#pragma unroll
          for (int t = 0; t < 8; t++)
#pragma unroll
            for (int c = 0; c < 4; c++) mx[c] = max(mx[c], abs_bits(y[t][c]));
          // column maxima of the eight warps meet in the (consumed) A staging
          uint32_t *part_max = reinterpret_cast<uint32_t *>(smem + a * L::kStgBytes);
#pragma unroll
          for (int c = 0; c < 4; c++) part_max[w * 128 + l + 32 * c] = mx[c];
          work_sync();
#pragma unroll
          for (int c = 0; c < 4; c++) {
            uint32_t m8 = 0;
#pragma unroll
            for (int ww = 0; ww < kFWorkers / 32; ww++) m8 = max(m8, part_max[ww * 128 + l + 32 * c]);
            sc[c] = scale_exponent(m8);
          }
        }
        if (w == 0) {
#pragma unroll
          for (int c = 0; c < 4; c++) sb[l + 32 * c] = (int16_t)sc[c];
        }
#pragma unroll
        for (int c = 0; c < 4; c++) {
          if (!col_in[c]) continue;
          uint2 lo[PARTS], hi[PARTS];
          split4f<PARTS>(make_float4(y[0][c], y[1][c], y[2][c], y[3][c]), scaled, sc[c], lo);
          split4f<PARTS>(make_float4(y[4][c], y[5][c], y[6][c], y[7][c]), scaled, sc[c], hi);
          const int jr = l + 32 * c;  // row of the K-major B operand
#pragma unroll
          for (int pp = 0; pp < PARTS; pp++)
            *reinterpret_cast<uint4 *>(op_b + pp * L::kPartBytes + swz(jr, 2 * w)) =
                make_uint4(lo[pp].x, lo[pp].y, hi[pp].x, hi[pp].y);
        }
        if (wt == 0) flags[1] = scaled ? 1 : 0;
      }
      fence_async_smem();  // the generic-proxy writes, before the MMAs read them
      mbar_arrive(opnd_full);
      // every worker is done with staging buffer a: refill it
      work_sync();
      if (wt == 0 && issued < nkb) {
        fence_async_smem();
        issue_stage(issued);
        issued++;
      }
      // the previous block's partial product, while this block's MMAs run
      if (j >= 1 && !accumulate(j - 1)) {
        ok = false;
        break;
      }
    }
    if (ok && nkb >= 1 && !accumulate(nkb - 1)) ok = false;
    if (wt == 0) {
      // loads still in flight after a timeout must land before the CTA's
      // shared memory goes away
      for (int jj = j; jj < issued; jj++)
        mbar_wait(stage_full(jj & 1), (uint32_t)((jj >> 1) & 1), err, 11, false, kFDrainNs);
    }
    // the partial row goes to the reduction buffer, which overlays the
    // staging buffers: every TMA load has landed and every block has been
    // converted once all roles meet here
    asm volatile("barrier.sync 3, %0;" ::"r"(kFThreads) : "memory");
    fence_async_smem();
    float *red = reinterpret_cast<float *>(smem);
#pragma unroll
    for (int c = 0; c < kFBN / 2; c++) red[row * kFRedPitch + ch * (kFBN / 2) + c] = acc[c];
  } else {
    if (lane == 0) {
      // ------------------------------------------------------------ MMA
      const uint32_t idesc = make_idesc<kTcSplitBf16x3>(kFBN);  // bf16 x bf16 -> f32, N = 128
      const uint32_t op = sbase + (uint32_t)L::kOpndOff;
      const uint32_t opb = op + PARTS * L::kPartBytes;
      bool issued = false, ok = true;
      for (int j = 0; j < nkb; j++) {
        const int a = j & 1;
        if (!mbar_wait(opnd_full, (uint32_t)(j & 1), err, 12, true, kFWaitNs)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(a * kFBN);
#pragma unroll
        for (int kk = 0; kk < kFBK / 16; kk++) {
          const uint64_t adv = (uint64_t)(kk * 32) >> 4;  // 16 bf16 = 32 bytes per MMA
          const uint32_t acc_in = kk != 0 ? 1u : 0u;
          const uint64_t a0 = kmajor_desc<128>(op) + adv, b0 = kmajor_desc<128>(opb) + adv;
          const uint64_t a1 = kmajor_desc<128>(op + L::kPartBytes) + adv;
          const uint64_t b1 = kmajor_desc<128>(opb + L::kPartBytes) + adv;
          if (PARTS == 2) {
            tc_mma(d_tmem, a0, b0, idesc, acc_in);  // hi.hi
            tc_mma(d_tmem, a0, b1, idesc, 1u);      // hi.lo
            tc_mma(d_tmem, a1, b0, idesc, 1u);      // lo.hi
          } else {
            // hi/mid/lo: products of relative size >= 2^-16, smallest first
            const uint64_t a2 = kmajor_desc<128>(op + 2 * L::kPartBytes) + adv;
            const uint64_t b2 = kmajor_desc<128>(opb + 2 * L::kPartBytes) + adv;
            tc_mma(d_tmem, a1, b1, idesc, acc_in);  // mid.mid
            tc_mma(d_tmem, a0, b2, idesc, 1u);      // hi.lo
            tc_mma(d_tmem, a2, b0, idesc, 1u);      // lo.hi
            tc_mma(d_tmem, a0, b1, idesc, 1u);      // hi.mid
            tc_mma(d_tmem, a1, b0, idesc, 1u);      // mid.hi
            tc_mma(d_tmem, a0, b0, idesc, 1u);      // hi.hi
          }
        }
        issued = true;
        tc_commit(acc_full(a));
        tc_commit(opnd_empty);
      }
      if (!ok && issued) {
        tc_commit(drain_bar);
        mbar_wait(drain_bar, 0, err, 12, false, kFDrainNs);
      }
    }
    asm volatile("barrier.sync 3, %0;" ::"r"(kFThreads) : "memory");
  }

  // ------------------------------------------------------------ reduction
  // Every thread of every CTA reaches this point (all waits are bounded), so
  // the cluster barriers below always complete.
  __syncthreads();
  float *red = reinterpret_cast<float *>(smem);  // [128][kFRedPitch]
  const int R = kTcBM / cs;  // rows of this CTA's chunk
  const int r0 = crank * R;
  const int64_t rows_left = (int64_t)pr.n - (row0 + r0);
  const int rows_valid = rows_left <= 0 ? 0 : (rows_left < R ? (int)rows_left : R);
  const int64_t cols_left = (int64_t)pr.p - col0;
  const int cols_valid = cols_left < kFBN ? (int)cols_left : kFBN;
  if (cs > 1) {
    cluster_sync_all();  // every rank's partial is in its shared memory
    // the ranks' buffers through distributed shared memory, rank order fixed
    namespace cgr = cooperative_groups;
    cgr::cluster_group cl = cgr::this_cluster();
    const float *rk_red[8];
#pragma unroll
    for (int rk = 0; rk < 8; rk++) rk_red[rk] = cl.map_shared_rank(red, rk < cs ? rk : 0);
    // four entries per thread at a time, all their loads in flight together
    for (int e0 = threadIdx.x; e0 < rows_valid * kFBN; e0 += 4 * kFThreads) {
      int off[4];
      float v[4][8];
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const int e = min(e0 + u * kFThreads, rows_valid * kFBN - 1);
        off[u] = (r0 + e / kFBN) * kFRedPitch + e % kFBN;
#pragma unroll
        for (int rk = 0; rk < 8; rk++) v[u][rk] = rk < cs ? rk_red[rk][off[u]] : 0.0f;
      }
      __syncwarp();
#pragma unroll
      for (int u = 0; u < 4; u++) {
        float sum = v[u][0];
#pragma unroll
        for (int rk = 1; rk < 8; rk++)
          if (rk < cs) sum += v[u][rk];
        if (e0 + u * kFThreads < rows_valid * kFBN) red[off[u]] = sum;  // own chunk rows only
      }
    }
    cluster_sync_all();  // no rank leaves while another may still read it
  } else {
    __syncthreads();
  }
  const bool failed = *reinterpret_cast<volatile int *>(err) != 0;
  const int nvalid = rows_valid * cols_valid;  // entries of this CTA's chunk inside C
  if (nvalid > 0 && !failed) {
    if (pr.Q == 1) {
      if (pr.epi.on == 0) {
        for (int e = threadIdx.x; e < nvalid; e += kFThreads) {
          const int rr = r0 + e / cols_valid, c = e % cols_valid;
          __stcs(pr.C + (row0 + rr) * pr.p + col0 + c, red[rr * kFRedPitch + c]);
        }
      } else {
        // C = alpha (A.B) + beta D, eight entries a thread at a time: their
        // values of D are loaded before any of them is stored (D may be C)
        for (int e0 = threadIdx.x; e0 < nvalid; e0 += 8 * kFThreads) {
          float dv[8];
          int64_t idx[8];
#pragma unroll
          for (int u = 0; u < 8; u++) {
            const int e = min(e0 + u * kFThreads, nvalid - 1);
            idx[u] = (row0 + r0 + e / cols_valid) * pr.p + col0 + e % cols_valid;
            dv[u] = pr.epi.on == 2 ? pr.epi.D[idx[u]] : 0.f;
          }
#pragma unroll
          for (int u = 0; u < 8; u++) {
            const int e = e0 + u * kFThreads;
            if (e < nvalid) {
              const float x = red[(r0 + e / cols_valid) * kFRedPitch + e % cols_valid];
              __stcs(pr.C + idx[u], pr.epi.on == 2 ? fmaf(pr.epi.alpha, x, pr.epi.beta * dv[u])
                                                   : pr.epi.alpha * x);
            }
          }
        }
      }
    } else {
      // clusters of this tile meet in global memory: slot (tile, q), then the
      // cluster that counts last on this chunk adds slots 0..Q-1 in order
      constexpr size_t kSlot = (size_t)kTcBM * kFBN;
      float *slot0 = pr.slots + (size_t)tile * pr.Q * kSlot;
      float *mine = slot0 + (size_t)q * kSlot;
      for (int e = threadIdx.x; e < nvalid; e += kFThreads) {
        const int rr = r0 + e / cols_valid, c = e % cols_valid;
        __stcg(mine + rr * kFBN + c, red[rr * kFRedPitch + c]);
      }
      __threadfence();
      __syncthreads();
      int *cnt = pr.cnt + (size_t)tile * cs + crank;
      if (threadIdx.x == 0) *last_flag = atomicAdd(cnt, 1) == pr.Q - 1;
      __syncthreads();
      if (*last_flag) {
        __threadfence();
        // slots 0..Q-1 in order for four entries per thread at a time, four
        // slots ahead: sixteen loads in flight per thread
        for (int e0 = threadIdx.x; e0 < nvalid; e0 += 4 * kFThreads) {
          const float *src[4];
          float sum[4];
#pragma unroll
          for (int u = 0; u < 4; u++) {
            const int e = min(e0 + u * kFThreads, nvalid - 1);
            src[u] = slot0 + (size_t)(r0 + e / cols_valid) * kFBN + e % cols_valid;
            sum[u] = __ldcg(src[u]);
          }
          // the epilogue's D for the same entries, in flight with the slots
          float dv[4];
          int64_t idx[4];
#pragma unroll
          for (int u = 0; u < 4; u++) {
            const int e = min(e0 + u * kFThreads, nvalid - 1);
            idx[u] = (row0 + r0 + e / cols_valid) * pr.p + col0 + e % cols_valid;
            dv[u] = pr.epi.on == 2 ? pr.epi.D[idx[u]] : 0.f;
          }
          int qq = 1;
          for (; qq + 4 <= pr.Q; qq += 4) {
            float v[4][4];
#pragma unroll
            for (int t = 0; t < 4; t++)
#pragma unroll
              for (int u = 0; u < 4; u++) v[t][u] = __ldcg(src[u] + (size_t)(qq + t) * kSlot);
#pragma unroll
            for (int t = 0; t < 4; t++)
#pragma unroll
              for (int u = 0; u < 4; u++) sum[u] += v[t][u];
          }
          for (; qq < pr.Q; qq++) {
#pragma unroll
            for (int u = 0; u < 4; u++) sum[u] += __ldcg(src[u] + (size_t)qq * kSlot);
          }
#pragma unroll
          for (int u = 0; u < 4; u++) {
            const int e = e0 + u * kFThreads;
            if (e < nvalid)
              __stcs(pr.C + idx[u], pr.epi.on == 0 ? sum[u]
                                    : pr.epi.on == 2 ? fmaf(pr.epi.alpha, sum[u], pr.epi.beta * dv[u])
                                                     : pr.epi.alpha * sum[u]);
          }
        }
        if (threadIdx.x == 0) *cnt = 0;  // ready for the next launch
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == kFMma) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem_base, kFTmemCols);
  }
}

}  // namespace
// ---------------------------------------------------------------- host side
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

// 2-D FP32 map over a row-major rows x cols matrix (row pitch cols * 4 bytes,
// a multiple of 16), boxes of box_cols x box_rows; reads outside the matrix
// return zero.
cudaError_t encode_f32_map(CUtensorMap *map, const float *base, int64_t rows, int64_t cols,
                           int box_cols, int box_rows) {
  auto enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * 4};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides,
                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int PARTS>
cudaError_t fused_attr() {
  static std::once_flag once;
  static cudaError_t e = cudaSuccess;
  std::call_once(once, [] {
    e = cudaFuncSetAttribute(tc_fused_kernel<PARTS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             FusedLayout<PARTS>::kSmemBytes);
  });
  return e;
}

template <int PARTS>
cudaError_t launch_fused_t(const FusedProb &pr, int cs, int *d_err, cudaStream_t s) {
  using L = FusedLayout<PARTS>;
  static_assert(L::kSmemBytes <= 232448, "shared memory budget");
  cudaError_t e = fused_attr<PARTS>();
  if (e != cudaSuccess) return e;
  CUtensorMap map_a, map_b;
  e = encode_f32_map(&map_a, pr.A, pr.n, pr.m, kFBK, kTcBM);
  if (e == cudaSuccess) e = encode_f32_map(&map_b, pr.B, pr.m, pr.p, kFBN, kFBK);
  if (e != cudaSuccess) return e;
  const int64_t ctas = (int64_t)pr.mt * pr.nt * pr.S;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)ctas, 1, 1);
  cfg.blockDim = dim3(kFThreads, 1, 1);
  cfg.dynamicSmemBytes = L::kSmemBytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = (unsigned)cs;
  attr[1].val.clusterDim.y = 1;
  attr[1].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = cs > 1 ? 2 : 1;
  TraceScope ts("fused_tc", s);
  return cudaLaunchKernelEx(&cfg, tc_fused_kernel<PARTS>, map_a, map_b, pr, d_err);
}

template <int PARTS>
int capacity_t(int cs) {
  static std::once_flag once;
  static int cap[4] = {0, 0, 0, 0};
  std::call_once(once, [] {
    if (fused_attr<PARTS>() != cudaSuccess) return;
    for (int k = 0; k < 4; k++) {
      const int c = 1 << k;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)(c * 64), 1, 1);
      cfg.blockDim = dim3(kFThreads, 1, 1);
      cfg.dynamicSmemBytes = FusedLayout<PARTS>::kSmemBytes;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = (unsigned)c;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int clusters = 0;
      if (cudaOccupancyMaxActiveClusters(&clusters, tc_fused_kernel<PARTS>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        clusters = 0;
      }
      cap[k] = clusters * c;
    }
  });
  const int k = cs >= 8 ? 3 : (cs >= 4 ? 2 : (cs >= 2 ? 1 : 0));
  return cap[k];
}

}  // namespace

bool fused_operands_ok(const float *A, const float *B, int64_t m, int64_t p) {
  return (reinterpret_cast<uintptr_t>(A) & 15u) == 0 && (reinterpret_cast<uintptr_t>(B) & 15u) == 0 &&
         (m & 3) == 0 && (p & 3) == 0;
}

cudaError_t launch_fused(bool six, const FusedProb &pr, int cs, int *d_err, cudaStream_t s) {
  if (cs != 1 && cs != 2 && cs != 4 && cs != 8) return cudaErrorInvalidValue;
  if (pr.S <= 0 || pr.Q <= 0 || pr.S % pr.Q != 0 || pr.S / pr.Q != cs) return cudaErrorInvalidValue;
  if (!fused_operands_ok(pr.A, pr.B, pr.m, pr.p)) return cudaErrorInvalidValue;
  return six ? launch_fused_t<3>(pr, cs, d_err, s) : launch_fused_t<2>(pr, cs, d_err, s);
}

int fused_capacity(bool six, int cs) { return six ? capacity_t<3>(cs) : capacity_t<2>(cs); }

}  // namespace mm
