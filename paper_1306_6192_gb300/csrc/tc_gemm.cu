// Tensor-core GEMM on sm_103a (tcgen05 + TMA + TMEM) for the FP32-in/out
// paths that run on the tensor cores.
//
// Split-BF16x3 kind: computes C = A.B for FP32 A, B, C from the packed bf16
// hi/lo operands written by split_prep.cu:
//     C_ij ~= 2^(s_i + t_j) * sum_r (Ah Bh + Ah Bl + Al Bh)_irj
// accumulated in FP32 in tensor memory; the lo.lo product (below 2^-16
// relative) is dropped.
// E4M3 kind: one e4m3 x e4m3 product per K step of the digit packs of the
// FP64 emulation (ozaki.cu), whose level products read windows of a longer
// pack through a per-problem K stride (a_kstride, b_kstride) and keep their
// integer sums exact in FP32.  (The FP32 FP8 mode has its own kernel with
// per-block scales, fp8_blk.cu.)
// The definition of the product is the paper's (Section "Implementacje
// algorytmow", Cauchy product); the split-precision method, the FP8 variant
// and everything below are this library's GB300 design, not the paper's (its
// kernels, Listings 2-4, use CUDA cores only).
//
// Kernel structure (persistent, one CTA per SM, 192 threads):
//   warp 0    TMEM allocation; lane 0 issues TMA loads of the A and B pack
//             tiles (all parts) of each K step into a STAGES-deep shared-
//             memory ring (mbarrier "full" with transaction bytes).
//   warp 1    lane 0 issues tcgen05.mma (M = 128, N = bn, 32 bytes of K per
//             instruction) - three per K step for the split kind, one for
//             e4m3 - and commits each stage back to the producer ("empty")
//             and each finished tile to the epilogue ("acc_full").
//   warps 2-5 epilogue: tcgen05.ld of the accumulator (each warp reads its
//             32 TMEM lanes = 32 rows), exact power-of-two unscaling, each
//             32 x 32 block through shared memory: one tiled TMA store per
//             block where the host gave C a tensor map (the store clips the
//             edges), else whole 128-byte-line stores of each row (edge rows
//             and columns predicated); then "acc_empty".
// Two accumulators of 256 TMEM columns each (four of 128 in the 128-wide
// layouts) let the epilogue of one tile overlap the mainloop of the next.
// The work units (tiles, or K parts of split tiles) of all problems of a
// table are visited in a static stride over the CTAs, the tiles of a problem
// in bands of group_m row tiles for L2 reuse.
// Tail split: where a product's tile count leaves the last wave of the
// persistent grid partly empty, the host cuts that product's last tiles into
// split_s parts along K (a plan fixed by the product's own shape, so a
// product gets the same bits alone and in any table).  Each part is a work
// unit of its own; its epilogue writes the FP32 partial tile to scratch and
// counts itself on the tile's counter, and the part that arrives last adds
// the parts in the fixed order 0..split_s-1 (its own from TMEM) before the
// usual unscaling and store, so the result does not depend on which part
// finishes first.  No CTA waits for another.
//
// Every mbarrier wait is bounded (kWaitLimitNs); on expiry a device flag is
// set, the other roles stop at their next wait, in-flight copies and MMAs
// are drained (bounded again) and TMEM is freed before the CTA exits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <utility>
#include <vector>

#include "tc_ptx.cuh"

namespace mm {
namespace {

constexpr int kThreads = 192;
constexpr uint32_t kTmemCols = 512;         // all of TMEM: the accumulators
constexpr int kBoxRows = 128;               // TMA box height (rows of the pack)
constexpr int kMaxSplit = 4;                // most K parts of a tail-split tile
constexpr uint64_t kWaitLimitNs = 4000000000ull;
constexpr uint64_t kDrainLimitNs = 200000000ull;

using namespace tcx;

// AND of `v` over the 128 epilogue threads (named barrier 1): every thread
// arrives, so the four warps leave the tile loop together.
__device__ __forceinline__ bool epilogue_all(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.and.pred p, 1, 128, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
}

// Power-of-two exponent applied to a row/column in the epilogue: the split
// path scales to max |x 2^-s| in [1, 2); the e4m3 path to [128, 256), which
// stays below the e4m3 maximum 448 and keeps 13 binades above its subnormals.
template <int KIND>
__device__ __forceinline__ int kind_exponent(uint32_t max_bits) {
  const int e = scale_exponent(max_bits);
  if (KIND != kTcE4m3) return e;
  const float f = __uint_as_float(max_bits);
  return (f > 0.0f && f <= 3.402823466e38f) ? e - 7 : 0;
}

// Work unit u of a table: problem g, output tile (mt, nt) = local tile t of
// the problem in raster order (bands of group_m row tiles), and part h of a
// tile split along K (h = -1: the whole tile).
struct UnitCoord {
  int g, mt, nt, t, h;
};

__device__ __forceinline__ UnitCoord decode_unit(const SplitProb *__restrict__ probs, int nprobs,
                                                 const int *__restrict__ map, int u) {
  const int g =
      find_problem(probs, nprobs, map, u, [](const SplitProb &q) { return q.unit_start; });
  const SplitProb &pr = probs[g];
  int t = u - pr.unit_start, h = -1;
  if (pr.split_s > 1 && t >= pr.split_from) {
    const int v = t - pr.split_from;
    t = pr.split_from + v / pr.split_s;
    h = v % pr.split_s;
  }
  const int gm = pr.group_m;
  const int band = gm * pr.nt;
  const int first = (t / band) * gm;
  const int rows = min(pr.mt - first, gm);
  const int in = t % band;
  return UnitCoord{g, first + in % rows, in / rows, t, h};
}

// FP8 tables with per-block factors: tile (mt, nt) of 128 x 256 keeps one
// exponent per row and column along K when its row tile and both of its
// 128-column halves are flagged (pr.cnt: mt row-tile flags, then the flags of
// the 128-column sub-tiles).  With uniform_only, the other tiles are skipped
// by every role (the blockwise kernel computes them).
__device__ __forceinline__ bool skip_unit(const SplitProb &pr, int uniform_only, int mt, int nt) {
  if (!uniform_only) return false;
  const int *f = pr.cnt;
  return !(f[mt] != 0 && f[pr.mt + 2 * nt] != 0 && f[pr.mt + 2 * nt + 1] != 0);
}

// Pipeline stages [k0, k1) of a unit: all kiters of a whole tile; for part h
// the stages of pack rows [h*kt/S, (h+1)*kt/S), so the split points do not
// depend on the stage depth BKB.
template <int BKB>
__device__ __forceinline__ void unit_krange(const SplitProb &pr, int h, int kiters, int &k0,
                                            int &k1) {
  if (h < 0) {
    k0 = 0;
    k1 = kiters;
    return;
  }
  constexpr int kStagesPerRow = kPackRowBytes / BKB;
  k0 = (int)((int64_t)h * pr.kt / pr.split_s) * kStagesPerRow;
  k1 = min((int)((int64_t)(h + 1) * pr.kt / pr.split_s) * kStagesPerRow, kiters);
}

__device__ __forceinline__ void epilogue_sync() {
  asm volatile("bar.sync 1, 128;" ::: "memory");
}

// Shared-memory layout of one instantiation: STAGES ring stages of BKB bytes
// of K for A (128 rows) and B (up to MAXBN rows) in every part.  Tables whose
// widest N tile is 128 take MAXBN = 128 layouts, whose smaller stages leave
// room for a deeper ring (small products have short K loops and need more
// loads in flight to cover the TMA latency).
template <int BKB, int STAGES, int KIND, int MAXBN>
struct TcLayout {
  static constexpr int kMaxBN = MAXBN;
  static constexpr int kParts = KIND == kTcE4m3 ? 1 : (KIND == kTcSplitBf16x3 ? 2 : 3);
  static constexpr int kElemBytes = KIND == kTcE4m3 ? 1 : 2;
  static constexpr int kAPart = kTcBM * BKB;            // one part of A per stage
  static constexpr int kBPartMax = kMaxBN * BKB;        // one part of B at bn = MAXBN
  static constexpr int kStageBytes = kParts * (kAPart + kBPartMax);
  static constexpr int kBarOffset = STAGES * kStageBytes;
  // accumulators of MAXBN TMEM columns: two at MAXBN = 256, four at 128, so
  // that the epilogues of short tiles can lag the MMAs by several tiles
  static constexpr int kNumAcc = (int)kTmemCols / kMaxBN;
  static constexpr int kNumBars = 2 * STAGES + 2 * kNumAcc + 1;  // full, empty, acc f/e, drain
  static constexpr int kColExpOffset = kBarOffset + kNumBars * 8 + 16;  // int[kNumAcc][kMaxBN]
  static constexpr int kLastOffset = kColExpOffset + kNumAcc * kMaxBN * 4;  // last-part flag
  // epilogue staging: one 32 x 33 float block per epilogue warp
  // epilogue staging, one 5 KB region per epilogue warp (1024-byte aligned):
  // a dense 32 x 32 FP32 block with a 128-byte swizzle for the tiled stores,
  // or rows of 33 floats for the plain stores
  static constexpr int kStageStride = 5120;
  static constexpr int kStageOffset = (kLastOffset + 16 + 1023) & ~1023;
  static constexpr int kSmemBytes = kStageOffset + 4 * kStageStride + 1024;  // + align slack
};

template <int BKB, int STAGES, int KIND, int MAXBN>
__global__ void __launch_bounds__(kThreads, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap tmap, const SplitProb *__restrict__ probs,
               int nprobs, const int *__restrict__ unit_map, const int *__restrict__ flags,
               int total_units, const int *__restrict__ order, int uniform_only,
               const CUtensorMap *__restrict__ c_maps, int *err) {
  using L = TcLayout<BKB, STAGES, KIND, MAXBN>;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t sbase = (raw + 1023u) & ~1023u;
  uint8_t *smem = smem_raw + (sbase - raw);
  const uint32_t bars = sbase + L::kBarOffset;
  auto full_bar = [&](int s) { return bars + 8u * s; };
  auto empty_bar = [&](int s) { return bars + 8u * (STAGES + s); };
  auto accf_bar = [&](int a) { return bars + 8u * (2 * STAGES + a); };
  auto acce_bar = [&](int a) { return bars + 8u * (2 * STAGES + L::kNumAcc + a); };
  const uint32_t drain_bar = bars + 8u * (2 * STAGES + 2 * L::kNumAcc);
  uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(smem + L::kBarOffset + L::kNumBars * 8);
  int *colexp = reinterpret_cast<int *>(smem + L::kColExpOffset);  // [kNumAcc][MAXBN]
  volatile int *last_flag = reinterpret_cast<volatile int *>(smem + L::kLastOffset);
  float *stage_buf = reinterpret_cast<float *>(smem + L::kStageOffset);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // this CTA's work units, the same sequence for every role: the host's list
  // (grid + 1 offsets, then the units), or units c, c + grid, ...
  const int *ulist = order ? order + gridDim.x + 1 : nullptr;
  const int i_first = order ? order[blockIdx.x] : (int)blockIdx.x;
  const int i_end = order ? order[blockIdx.x + 1] : total_units;
  const int i_step = order ? 1 : (int)gridDim.x;

  if (warp == 0) {
    tmem_alloc(smem_u32(tmem_holder), kTmemCols);
    tmem_relinquish();
  }
  if (threadIdx.x == 32) {
    for (int s = 0; s < STAGES; s++) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int a = 0; a < L::kNumAcc; a++) {
      mbar_init(accf_bar(a), 1);
      mbar_init(acce_bar(a), 4 * 32);
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
      // ------------------------------------------------------ TMA producer
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap))
                   : "memory");
      int stage = 0;
      uint32_t phase = 0;
      uint32_t issued = 0;  // stage loads armed so far
      bool ok = true;
      for (int ui = i_first; ui < i_end && ok; ui += i_step) {
        const int u = ulist ? ulist[ui] : ui;
        const UnitCoord tc = decode_unit(probs, nprobs, unit_map, u);
        const SplitProb &pr = probs[tc.g];
        if (skip_unit(pr, uniform_only, tc.mt, tc.nt)) continue;
        const int bn = pr.bn;
        const int kiters = (int)(((int64_t)pr.m * L::kElemBytes + BKB - 1) / BKB);
        const uint32_t bytes = (uint32_t)(L::kParts * (kTcBM + bn) * BKB);
        int k0, k1;
        unit_krange<BKB>(pr, tc.h, kiters, k0, k1);
        // first pack rows of the unit's A and B tiles (K block 0)
        const int64_t ak = pr.a_kstride > 0 ? pr.a_kstride : pr.kt;
        const int64_t bk = pr.b_kstride > 0 ? pr.b_kstride : pr.kt;
        const int64_t abase = pr.a_row0 + (int64_t)tc.mt * ak * (L::kParts * kTcBM);
        const int64_t bbase = pr.b_row0 + (int64_t)tc.nt * bk * (L::kParts * bn);
        for (int ki = k0; ki < k1; ki++) {
          if (!mbar_wait(empty_bar(stage), phase ^ 1u, err, 1, true, kWaitLimitNs)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(full_bar(stage), bytes);
          ++issued;
          const int kb = (ki * BKB) / kPackRowBytes;
          const int x = (ki * BKB) % kPackRowBytes;  // byte offset in the pack row
          const int64_t arow = abase + (int64_t)kb * (L::kParts * kTcBM);
          const int64_t brow = bbase + (int64_t)kb * (L::kParts * bn);
          const uint32_t st = sbase + stage * L::kStageBytes;
#pragma unroll
          for (int part = 0; part < L::kParts; part++)
            tma_load_2d(st + part * L::kAPart, &tmap, x, (int)(arow + part * kTcBM),
                        full_bar(stage));
          // B: parts * bn rows, a multiple of the 128-row box (tc_bn keeps
          // bn >= 128 unless parts = 2), so the boxes carry exactly the bytes
          // expected
          const uint32_t sb = st + L::kParts * L::kAPart;
          for (int r = 0; r < L::kParts * bn; r += kBoxRows)
            tma_load_2d(sb + r * BKB, &tmap, x, (int)(brow + r), full_bar(stage));
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (!ok) {
        // drain copies still in flight before the CTA's shared memory goes
        // away: the last STAGES loads armed, one per stage, load j in stage
        // j % STAGES with parity (j / STAGES) & 1
        for (uint32_t j = issued > STAGES ? issued - STAGES : 0; j < issued; j++)
          mbar_wait(full_bar((int)(j % STAGES)), (j / STAGES) & 1u, err, 1, false, kDrainLimitNs);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ------------------------------------------------------ MMA issuer
      int stage = 0;
      uint32_t phase = 0;
      int acc = 0;
      uint32_t acc_phase = 0;
      bool ok = true, issued = false;
      for (int ui = i_first; ui < i_end && ok; ui += i_step) {
        const int u = ulist ? ulist[ui] : ui;
        const UnitCoord tc = decode_unit(probs, nprobs, unit_map, u);
        const SplitProb &pr = probs[tc.g];
        if (skip_unit(pr, uniform_only, tc.mt, tc.nt)) continue;
        const int kiters = (int)(((int64_t)pr.m * L::kElemBytes + BKB - 1) / BKB);
        int k0, k1;
        unit_krange<BKB>(pr, tc.h, kiters, k0, k1);
        const uint32_t idesc = make_idesc<KIND>(pr.bn);
        const uint32_t blo = (uint32_t)pr.bn * BKB;
        if (!mbar_wait(acce_bar(acc), acc_phase ^ 1u, err, 2, true, kWaitLimitNs)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(acc * MAXBN);
        for (int ki = k0; ki < k1; ki++) {
          if (!mbar_wait(full_bar(stage), phase, err, 3, true, kWaitLimitNs)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t st = sbase + stage * L::kStageBytes;
          const uint32_t sb = st + L::kParts * L::kAPart;
          const uint64_t a0 = kmajor_desc<BKB>(st);
          const uint64_t b0 = kmajor_desc<BKB>(sb);
#pragma unroll
          for (int kk = 0; kk < BKB / 32; kk++) {
            // 32 bytes of K per instruction: 16 bf16 or 32 e4m3
            const uint64_t adv = (uint64_t)(kk * 32) >> 4;
            const uint32_t acc_in = (ki != k0 || kk != 0) ? 1u : 0u;
            if (KIND == kTcSplitBf16x3) {
              const uint64_t a1 = kmajor_desc<BKB>(st + L::kAPart);
              const uint64_t b1 = kmajor_desc<BKB>(sb + blo);
              tc_mma(d_tmem, a0 + adv, b0 + adv, idesc, acc_in);  // hi.hi
              tc_mma(d_tmem, a0 + adv, b1 + adv, idesc, 1u);      // hi.lo
              tc_mma(d_tmem, a1 + adv, b0 + adv, idesc, 1u);      // lo.hi
            } else if (KIND == kTcSplitBf16x6) {
              // parts 0/1/2 = hi/mid/lo; products of relative size >= 2^-16,
              // smallest first
              const uint64_t a1 = kmajor_desc<BKB>(st + L::kAPart);
              const uint64_t a2 = kmajor_desc<BKB>(st + 2 * L::kAPart);
              const uint64_t b1 = kmajor_desc<BKB>(sb + blo);
              const uint64_t b2 = kmajor_desc<BKB>(sb + 2 * blo);
              tc_mma(d_tmem, a1 + adv, b1 + adv, idesc, acc_in);  // mid.mid
              tc_mma(d_tmem, a0 + adv, b2 + adv, idesc, 1u);      // hi.lo
              tc_mma(d_tmem, a2 + adv, b0 + adv, idesc, 1u);      // lo.hi
              tc_mma(d_tmem, a0 + adv, b1 + adv, idesc, 1u);      // hi.mid
              tc_mma(d_tmem, a1 + adv, b0 + adv, idesc, 1u);      // mid.hi
              tc_mma(d_tmem, a0 + adv, b0 + adv, idesc, 1u);      // hi.hi
            } else {
              tc_mma_f8(d_tmem, a0 + adv, b0 + adv, idesc, acc_in);
            }
          }
          issued = true;
          tc_commit(empty_bar(stage));
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        tc_commit(accf_bar(acc));
        if (++acc == L::kNumAcc) {
          acc = 0;
          acc_phase ^= 1u;
        }
      }
      if (!ok && issued) {
        // wait for MMAs in flight before TMEM is released
        tc_commit(drain_bar);
        mbar_wait(drain_bar, 0, err, 3, false, kDrainLimitNs);
      }
    }
  } else {
    // -------------------------------------------------------- epilogue
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    const int row = q * 32 + lane;
    int acc = 0;
    uint32_t acc_phase = 0;
    const int et = threadIdx.x - 64;  // 0..127 over the epilogue warps
    for (int ui = i_first; ui < i_end; ui += i_step) {
      const int u = ulist ? ulist[ui] : ui;
      const UnitCoord tc = decode_unit(probs, nprobs, unit_map, u);
      const SplitProb &pr = probs[tc.g];
      if (skip_unit(pr, uniform_only, tc.mt, tc.nt)) continue;
      // column exponents of this tile, once per tile, while the MMAs run
      // operands packed without scaling (flags) take exponent 0
      const int fl = flags ? flags[tc.g] : (kFlagScaleA | kFlagScaleB);
      int *cexp = colexp + acc * MAXBN;
      for (int c = et; c < pr.bn; c += 128) {
        const int64_t j = (int64_t)tc.nt * pr.bn + c;
        cexp[c] = (j < pr.p && (fl & kFlagScaleB)) ? kind_exponent<KIND>(pr.tB[j]) : 0;
      }
      const bool ok = mbar_wait(accf_bar(acc), acc_phase, err, 4, true, kWaitLimitNs);
      if (!epilogue_all(ok)) break;  // also orders the cexp writes before the reads
      tc_fence_after();
      const int64_t i = (int64_t)tc.mt * kTcBM + row;
      const bool row_ok = i < pr.n;
      const int si = (row_ok && (fl & kFlagScaleA)) ? kind_exponent<KIND>(pr.sA[i]) : 0;
      float *buf = stage_buf + q * (L::kStageStride / 4);  // this warp's 32 x 32 block
      const CUtensorMap *cmap = (c_maps != nullptr && pr.c_tma > 0) ? c_maps + (pr.c_tma - 1)
                                                                     : nullptr;
      const int64_t row0 = (int64_t)tc.mt * kTcBM + q * 32;  // first row of the warp
      const uint32_t tacc = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * MAXBN);
      // part of a split tile: a partial slot holds bn/4 groups of 4 columns,
      // each group 128 rows x 4 floats, so that a warp's 16-byte accesses to
      // one group (32 rows) are 512 consecutive bytes
      const size_t slot_floats = (size_t)kTcBM * pr.bn;
      const int split_s = pr.split_s;
      const int st = tc.t - pr.split_from;  // index among the split tiles
      const float4 *slots = tc.h >= 0 ? reinterpret_cast<const float4 *>(
                                            pr.part + (size_t)st * split_s * slot_floats) + row
                                      : nullptr;
      bool store = true;
      if (tc.h >= 0) {
        float4 *mine = reinterpret_cast<float4 *>(
                           pr.part + ((size_t)st * split_s + tc.h) * slot_floats) + row;
        for (int c = 0; c < pr.bn; c += 32) {
          uint32_t v[32];
          __syncwarp();
          tmem_ld_32x32b_x32(tacc + (uint32_t)c, v);
          tmem_ld_wait();
#pragma unroll
          for (int e = 0; e < 32; e += 4)
            __stcg(mine + (size_t)((c + e) >> 2) * kTcBM,
                   make_float4(__uint_as_float(v[e]), __uint_as_float(v[e + 1]),
                               __uint_as_float(v[e + 2]), __uint_as_float(v[e + 3])));
        }
        __threadfence();
        epilogue_sync();  // every row of this part written and fenced
        if (et == 0) *last_flag = atomicAdd(pr.cnt + st, 1) == split_s - 1;
        epilogue_sync();
        store = *last_flag != 0;
        if (store) {
          __threadfence();
          if (et == 0) pr.cnt[st] = 0;  // ready for the next launch
        }
      }
      for (int c = 0; c < pr.bn && store; c += 32) {
        uint32_t v[32];
        __syncwarp();  // tcgen05.ld is warp-collective: reconverge first
        tmem_ld_32x32b_x32(tacc + (uint32_t)c, v);
        tmem_ld_wait();
        if (tc.h >= 0) {
          // sum of the parts in order 0..split_s-1 (this part's from TMEM);
          // the loads of all other parts of the chunk are issued first
          float4 x[kMaxSplit][8];
#pragma unroll
          for (int hh = 0; hh < kMaxSplit; hh++) {
            if (hh < split_s && hh != tc.h) {
              const float4 *src = slots + (size_t)hh * (slot_floats / 4) + (size_t)(c >> 2) * kTcBM;
#pragma unroll
              for (int e = 0; e < 8; e++) x[hh][e] = __ldcg(src + (size_t)e * kTcBM);
            }
          }
#pragma unroll
          for (int e = 0; e < 8; e++) {
            float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int hh = 0; hh < kMaxSplit; hh++) {
              if (hh >= split_s) break;
              const float4 y = hh == tc.h ? make_float4(__uint_as_float(v[4 * e]),
                                                        __uint_as_float(v[4 * e + 1]),
                                                        __uint_as_float(v[4 * e + 2]),
                                                        __uint_as_float(v[4 * e + 3]))
                                          : x[hh][e];
              if (hh == 0) {
                sum = y;
              } else {
                sum.x += y.x;
                sum.y += y.y;
                sum.z += y.z;
                sum.w += y.w;
              }
            }
            v[4 * e] = __float_as_uint(sum.x);
            v[4 * e + 1] = __float_as_uint(sum.y);
            v[4 * e + 2] = __float_as_uint(sum.z);
            v[4 * e + 3] = __float_as_uint(sum.w);
          }
        }
        const int64_t j0 = (int64_t)tc.nt * pr.bn + c;
        if (j0 >= pr.p) continue;  // the same for the whole warp
        const int *ce = cexp + c;
        if (cmap) {
          // the block into the dense staging area, 16-byte chunk k of row
          // `lane` at chunk k ^ (lane & 7) (the 128-byte swizzle of the map;
          // the writes of one instruction then spread over all banks), and
          // one tiled store of it; the area is rewritten only after the
          // previous store has read it
          if (lane == 0) bulk_wait_read_all();
          __syncwarp();
          float4 *rowp = reinterpret_cast<float4 *>(buf + lane * 32);
#pragma unroll
          for (int k = 0; k < 8; k++)
            rowp[k ^ (lane & 7)] =
                make_float4(scale_pow2(__uint_as_float(v[4 * k]), si + ce[4 * k]),
                            scale_pow2(__uint_as_float(v[4 * k + 1]), si + ce[4 * k + 1]),
                            scale_pow2(__uint_as_float(v[4 * k + 2]), si + ce[4 * k + 2]),
                            scale_pow2(__uint_as_float(v[4 * k + 3]), si + ce[4 * k + 3]));
          if (pr.epi.on != 0) {
            // C = alpha (A.B) + beta D on this thread's row of the block, in
            // place in the staging area: the row's 32 values of D in eight
            // 16-byte loads in flight (p % 4 == 0 and a 16-byte aligned D,
            // so a vector is wholly inside or outside C's columns)
            const int64_t i = row0 + lane;
            const float al = pr.epi.alpha, be = pr.epi.beta;
            if (pr.epi.on == 2) {
              const float4 *drow = reinterpret_cast<const float4 *>(pr.epi.D + i * pr.p + j0);
              float4 dq[8];
#pragma unroll
              for (int k = 0; k < 8; k++)
                dq[k] = (i < pr.n && j0 + 4 * k < pr.p) ? drow[k] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
              for (int k = 0; k < 8; k++) {
                const float4 x = rowp[k ^ (lane & 7)];
                rowp[k ^ (lane & 7)] = make_float4(fmaf(al, x.x, be * dq[k].x), fmaf(al, x.y, be * dq[k].y),
                                                   fmaf(al, x.z, be * dq[k].z), fmaf(al, x.w, be * dq[k].w));
              }
            } else {
#pragma unroll
              for (int k = 0; k < 8; k++) {
                const float4 x = rowp[k];
                rowp[k] = make_float4(al * x.x, al * x.y, al * x.z, al * x.w);
              }
            }
          }
          fence_proxy_async_shared();
          __syncwarp();
          if (lane == 0 && row0 < pr.n) {  // a block wholly below C is not stored
            tma_store_2d(cmap, smem_u32(buf), (int)j0, (int)row0);
            bulk_commit();
          }
          continue;
        }
        // unscale this thread's row of the 32 x 32 block into shared memory,
        // then write the block row by row: each store is 32 consecutive
        // columns of one row, a whole 128-byte line
#pragma unroll
        for (int e = 0; e < 32; e++)
          buf[lane * 33 + e] = scale_pow2(__uint_as_float(v[e]), si + ce[e]);
        __syncwarp();
        const int64_t j = j0 + lane;
        if (j < pr.p) {
          float *dst = pr.C + row0 * pr.p + j;
          const int64_t left = pr.n - row0;
          const int rows = left < 32 ? (int)left : 32;
          if (pr.epi.on == 0) {
#pragma unroll 8
            for (int r = 0; r < rows; r++, dst += pr.p) __stcs(dst, buf[r * 33 + lane]);
          } else {
            // C = alpha (A.B) + beta D, sixteen rows at a time: their values
            // of D are loaded before any of them is stored (D may be C)
            const float *dcol = pr.epi.D + row0 * pr.p + j;
#pragma unroll
            for (int h = 0; h < 32; h += 16) {
              float dv[16];
#pragma unroll
              for (int r = 0; r < 16; r++)
                dv[r] = (pr.epi.on == 2 && h + r < rows) ? dcol[(int64_t)(h + r) * pr.p] : 0.f;
#pragma unroll
              for (int r = 0; r < 16; r++)
                if (h + r < rows)
                  __stcs(dst + (int64_t)(h + r) * pr.p,
                         pr.epi.on == 2
                             ? fmaf(pr.epi.alpha, buf[(h + r) * 33 + lane], pr.epi.beta * dv[r])
                             : pr.epi.alpha * buf[(h + r) * 33 + lane]);
            }
          }
        }
        __syncwarp();
      }
      tc_fence_before();
      mbar_arrive(acce_bar(acc));
      if (++acc == L::kNumAcc) {
        acc = 0;
        acc_phase ^= 1u;
      }
    }
    // the tiled stores have read shared memory and completed
    if (lane == 0) bulk_wait_all();
    __syncwarp();
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem_base, kTmemCols);
  }
}

// ---------------------------------------------------------------- host side
PFN_cuTensorMapEncodeTiled_v12000 get_encode_fn() {
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

// 2-D map over the pack region viewed as rows of 128 bytes; a box is BKB
// bytes of 128 consecutive rows.
cudaError_t encode_pack_map(CUtensorMap *map, void *base, int64_t rows, int bkb) {
  auto enc = get_encode_fn();
  if (!enc) return cudaErrorNotSupported;
  cuuint64_t dims[2] = {(cuuint64_t)kPackRowBytes, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kPackRowBytes};
  cuuint32_t box[2] = {(cuuint32_t)bkb, (cuuint32_t)kBoxRows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, base, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE,
                   bkb == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

// 2-D map over C (n rows of p FP32, row-major) for the epilogue's tiled
// stores: boxes of 32 x 32 with a 128-byte swizzle.  Needs a 16-byte aligned
// C and p a multiple of 4.
bool tc_c_map_ok(const float *C, int64_t n, int64_t p) {
  return (reinterpret_cast<uintptr_t>(C) & 15u) == 0 && (p & 3) == 0 && n > 0 && p > 0 &&
         n <= 0x7fffffffLL && p <= 0x7fffffffLL;
}

cudaError_t encode_c_map(void *map, float *C, int64_t n, int64_t p) {
  auto enc = get_encode_fn();
  if (!enc) return cudaErrorNotSupported;
  cuuint64_t dims[2] = {(cuuint64_t)p, (cuuint64_t)n};
  cuuint64_t strides[1] = {(cuuint64_t)p * 4};
  cuuint32_t box[2] = {32u, 32u};
  cuuint32_t estr[2] = {1, 1};
  CUtensorMap tmp;  // 64-byte aligned; `map` need not be
  CUresult r = enc(&tmp, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, C, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  std::memcpy(map, &tmp, sizeof(tmp));
  return cudaSuccess;
}

namespace {

template <int BKB, int STAGES, int KIND, int MAXBN>
cudaError_t launch_tc_t(const SplitProb *d_probs, int nprobs, const int *unit_map,
                        const int *flags, int total_units, void *pack_base, int64_t pack_rows,
                        int grid, int *d_err, cudaStream_t s, const int *order,
                        int uniform_only, const void *c_maps) {
  using L = TcLayout<BKB, STAGES, KIND, MAXBN>;
  static_assert(L::kSmemBytes <= 232448, "shared memory budget");
  // one CTA per SM: the kernel allocates all 512 TMEM columns
  static_assert(2 * L::kSmemBytes > 232448, "must not fit twice on one SM");
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [] {
    attr_err = cudaFuncSetAttribute(tc_gemm_kernel<BKB, STAGES, KIND, MAXBN>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, L::kSmemBytes);
  });
  if (attr_err != cudaSuccess) return attr_err;
  CUtensorMap map;
  cudaError_t e = encode_pack_map(&map, pack_base, pack_rows, BKB);
  if (e != cudaSuccess) return e;
  TraceScope ts(KIND == kTcE4m3 ? "fp8_tc" : "split_tc", s);
  tc_gemm_kernel<BKB, STAGES, KIND, MAXBN><<<grid, kThreads, L::kSmemBytes, s>>>(
      map, d_probs, nprobs, unit_map, flags, total_units, order, uniform_only,
      static_cast<const CUtensorMap *>(c_maps), d_err);
  return cudaGetLastError();
}

}  // namespace

int tc_grid(const TcConfig &cfg) { return cfg.grid > 0 ? cfg.grid : sm_count(); }

int tc_launch_grid(const TcConfig &cfg, int64_t total_units) {
  const int g = tc_grid(cfg);
  return total_units < g ? (int)std::max<int64_t>(total_units, 1) : g;
}

void tc_unit_order(const SplitProb *tab, int nprobs, int grid, std::vector<int> &out) {
  int64_t total = 0;
  for (int g = 0; g < nprobs; g++) total += split_units(tab[g]);
  out.assign((size_t)grid + 1 + (size_t)total, 0);
  if (grid <= 0) return;
  // (expected free time, CTA): a binary heap on the earliest time, lowest CTA
  std::vector<std::pair<int64_t, int>> heap;
  heap.reserve((size_t)grid);
  for (int c = 0; c < grid; c++) heap.emplace_back(0, c);
  auto later = [](const std::pair<int64_t, int> &a, const std::pair<int64_t, int> &b) {
    return a.first != b.first ? a.first > b.first : a.second > b.second;
  };
  std::make_heap(heap.begin(), heap.end(), later);
  std::vector<int> owner((size_t)total);
  std::vector<int> count((size_t)grid, 0);
  for (int g = 0; g < nprobs; g++) {
    const SplitProb &pr = tab[g];
    const int64_t units = split_units(pr);
    for (int64_t t = 0; t < units; t++) {
      int64_t rows = pr.kt;  // K pack rows of the unit
      if (pr.split_s > 1 && t >= pr.split_from) {
        const int64_t h = (t - pr.split_from) % pr.split_s;
        rows = (h + 1) * pr.kt / pr.split_s - h * pr.kt / pr.split_s;
      }
      std::pop_heap(heap.begin(), heap.end(), later);
      auto &slot = heap.back();
      owner[(size_t)(pr.unit_start + t)] = slot.second;
      count[(size_t)slot.second]++;
      slot.first += rows + 1;
      std::push_heap(heap.begin(), heap.end(), later);
    }
  }
  int *off = out.data();
  for (int c = 0; c < grid; c++) off[c + 1] = off[c] + count[(size_t)c];
  std::vector<int> fill(off, off + grid);
  int *list = off + grid + 1;
  for (int64_t u = 0; u < total; u++) list[fill[(size_t)owner[(size_t)u]]++] = (int)u;
}

TcTail tc_tail_plan(int64_t tiles, int grid, int kt, int bn, int64_t m, double products) {
  TcTail best{(int)tiles, 1};
  if (tiles <= 0 || grid <= 1 || kt < 4) return best;
  const int64_t G = grid;
  if (tiles < G && kt < 16) return best;  // small products: grouped tables hold many
  // units c, c + G, c + 2G, ... below x go to CTA c
  auto upto = [G](int64_t x, int64_t c) -> int64_t { return x > c ? (x - c + G - 1) / G : 0; };
  // per-unit overhead of a part, in tiles: the pipeline refill (~2 us)
  // against a tile's time at the per-SM tensor rate (~12.8 TFLOP/s of bf16
  // products); the part that finishes a tile writes its partial and reads
  // the others, latency-bound while the other SMs load L2 (~40 GB/s per SM
  // measured for this pattern on GB300)
  const double tile_us = 2.0 * kTcBM * bn * (double)m * products / 12.8e6;
  const double eps = 0.01 + 2.0 / tile_us;
  const double slot_us = (double)kTcBM * bn * 4.0 / 40e3;
  auto makespan = [&](int64_t F, int S) {
    const int64_t U = F + (tiles - F) * S;
    double worst = 0.0;
    for (int64_t c = 0; c < G; c++) {
      const double cost =
          (double)upto(F, c) + (double)(upto(U, c) - upto(F, c)) * (1.0 / S + eps);
      worst = cost > worst ? cost : worst;
    }
    return S > 1 ? worst + S * slot_us / tile_us : worst;
  };
  double best_cost = makespan(tiles, 1);
  const int64_t rem = tiles % G;
  for (int64_t R : {rem, rem + G}) {
    if (R <= 0 || R > tiles) continue;
    for (int S = 2; S <= kMaxSplit && R * S <= 2 * G && kt / S >= 2; S++) {
      const double c = makespan(tiles - R, S);
      if (c < best_cost - 1e-9) {
        best_cost = c;
        best = TcTail{(int)(tiles - R), S};
      }
    }
  }
  return best;
}

size_t tc_tail_part_bytes(const TcTail &t, int64_t tiles, int bn) {
  if (t.split_s <= 1) return 0;
  const int64_t R = tiles - t.split_from;
  return ((size_t)R * t.split_s * kTcBM * bn * sizeof(float) + 255) & ~(size_t)255;
}

size_t tc_tail_bytes(const TcTail &t, int64_t tiles, int bn) {
  if (t.split_s <= 1) return 0;
  const int64_t R = tiles - t.split_from;
  return tc_tail_part_bytes(t, tiles, bn) + (((size_t)R * sizeof(int) + 255) & ~(size_t)255);
}

cudaError_t launch_tc(TcKind kind, const SplitProb *d_probs, int nprobs, int total_units,
                      const int *unit_map, const int *flags, void *pack_base, int64_t pack_rows,
                      const TcConfig &cfg, int *d_err, cudaStream_t s, const int *order,
                      int uniform_only, const void *c_maps) {
  if (total_units <= 0) return cudaSuccess;
  if (pack_rows <= 0 || pack_rows > 0x7fffffffLL) return cudaErrorInvalidValue;
  const int grid = tc_launch_grid(cfg, total_units);
  const int *mp = unit_map;
#define MM_TC_ARGS \
  d_probs, nprobs, mp, flags, total_units, pack_base, pack_rows, grid, d_err, s, order, \
      uniform_only, c_maps
  cudaError_t e = cudaErrorInvalidValue;
  const bool narrow = cfg.max_bn <= 128;  // every N tile of the table fits 128
  if (kind == kTcE4m3) e = launch_tc_t<128, 4, kTcE4m3, 256>(MM_TC_ARGS);
  else if (kind == kTcSplitBf16x6 && narrow) e = launch_tc_t<64, 4, kTcSplitBf16x6, 128>(MM_TC_ARGS);
  else if (cfg.bkb == 128 && narrow) e = launch_tc_t<128, 3, kTcSplitBf16x3, 128>(MM_TC_ARGS);
  else if (cfg.bkb == 128) e = launch_tc_t<128, 2, kTcSplitBf16x3, 256>(MM_TC_ARGS);
  else if (cfg.bkb == 64 && narrow) e = launch_tc_t<64, 6, kTcSplitBf16x3, 128>(MM_TC_ARGS);
  else if (cfg.bkb == 64 && cfg.stages == 3) e = launch_tc_t<64, 3, kTcSplitBf16x3, 256>(MM_TC_ARGS);
  else if (cfg.bkb == 64) e = launch_tc_t<64, 4, kTcSplitBf16x3, 256>(MM_TC_ARGS);
#undef MM_TC_ARGS
  return e;
}

}  // namespace mm
