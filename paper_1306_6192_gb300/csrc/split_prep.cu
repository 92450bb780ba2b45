// Split-BF16x3 operand preparation.
//
// Method: an FP32 operand x is written as x = 2^s (hi + lo + d) with
// hi = bf16_rn(x 2^-s), lo = bf16_rn(x 2^-s - hi) and |d| <= 2^-16 |x 2^-s|
// (three parts: hi + mid + lo, |d| <= 2^-24 |x 2^-s|)
// (G. Henry, P. T. P. Tang, A. Heinecke, "Leveraging the bfloat16 artificial
// intelligence datatype for higher-precision computations", ARITH 2019).  The
// power-of-two scale 2^s is chosen per row of A and per column of B from the
// largest magnitude of that row/column, so operands far from 1 keep all their
// significant bits in the bf16 range; scaling by 2^s is exact.  Not part of
// the paper, whose kernels compute in the input type directly.
//
// Kernels:
//   split_pack_kernel   one block per 128 x 64 tile of A or bn x 64 tile of
//                       B^T: scale, split, write the bf16 parts (hi, lo - or
//                       hi, mid, lo for the three-part split) of the pack
//                       (layout in mm_internal.h); zero outside the matrix
//                       so the tensor-core kernel needs no edge checks.
//
// The split path packs in one pass over A and B (kPackUnscaled): scaling by
// a power of two commutes with rounding to bf16 and with the FP32 sums as long
// as nothing leaves the normal range, so for rows/columns whose largest
// magnitude lies in [2^-40, 2^40] the unscaled split gives the same bits as
// the scaled one.  That pass also writes each tile's row/column maxima;
// split_verify_kernel reduces them to the maxima of whole rows/columns and
// flags, per problem, an operand with a row/column outside the range, and a
// second pack launch (kPackFix) re-packs only the flagged operands with their
// scales.  The epilogue applies 2^(s_i + t_j) only for flagged operands.
#include <algorithm>

#include "split_common.cuh"

namespace mm {
namespace {


__device__ __forceinline__ uint32_t abs_bits(float x) { return __float_as_uint(x) & 0x7fffffffu; }

__device__ __forceinline__ uint32_t umax(uint32_t a, uint32_t b) { return a > b ? a : b; }

__device__ __forceinline__ bool aligned16(const void *p) {
  return (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
}

// Splits four values scaled by 2^-s (SCALED; unscaled: s = 0, no multiply)
// into PARTS groups of four bf16 (two bf16x2 words each): part 0 = RN(y),
// part q = RN(y - part 0 - ... - part q-1).  Every remainder is exact in FP32
// (the difference of a float and its rounding to fewer bits), so y = sum of
// parts + d, |d| <= 2^(-8*PARTS) |y|.
template <int PARTS, bool SCALED>
__device__ __forceinline__ void split4(float4 x, int s, uint2 (&out)[PARTS]) {
  float y[4] = {x.x, x.y, x.z, x.w};
  if (SCALED) {
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

// max |x| over four values as a float bit pattern
__device__ __forceinline__ uint32_t max4_bits(float4 x) {
  return umax(umax(abs_bits(x.x), abs_bits(x.y)), umax(abs_bits(x.z), abs_bits(x.w)));
}

// Eight maxima over the 16 lanes of a half warp at once (v[t], t = 0..7, in
// every lane): each exchange round sends the half of the slots that the
// partner keeps, so 8 shuffles replace 4 per slot.  Returns, in every lane,
// the half-warp maximum of slot t = (lane >> 1) & 7 (lanes 2t and 2t + 1 of
// the half warp hold slot t).  Every lane of the warp must call it.
__device__ __forceinline__ uint32_t half_warp_max8(const uint32_t (&v)[8]) {
  const int lane = threadIdx.x & 31;
  const bool b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
  uint32_t w[4], u[2];
#pragma unroll
  for (int j = 0; j < 4; j++) {  // lanes with bit 3 clear keep slots 0-3
    const uint32_t send = b3 ? v[j] : v[j + 4], keep = b3 ? v[j + 4] : v[j];
    w[j] = umax(keep, __shfl_xor_sync(0xffffffffu, send, 8));
  }
#pragma unroll
  for (int j = 0; j < 2; j++) {  // w[j] holds slot j + 4 b3
    const uint32_t send = b2 ? w[j] : w[j + 2], keep = b2 ? w[j + 2] : w[j];
    u[j] = umax(keep, __shfl_xor_sync(0xffffffffu, send, 4));
  }
  const uint32_t send = b1 ? u[0] : u[1], keep = b1 ? u[1] : u[0];  // u[j]: slot j + 2 b2 + 4 b3
  const uint32_t t = umax(keep, __shfl_xor_sync(0xffffffffu, send, 2));
  return umax(t, __shfl_xor_sync(0xffffffffu, t, 1));
}

// One B pack tile (nt, kb) of split_pack_kernel: bn columns x 64 k,
// transposed through shared memory CW columns at a time.
template <int PARTS, int MODE, int CW>
__device__ __forceinline__ void pack_b_tile(const SplitProb &pr, int b, uint2 *__restrict__ pack,
                                            float (&tile)[kPackK][128 + 1], int tid) {
  constexpr int kQuads = kPackK / 4;                 // groups of four bf16 per pack row
  constexpr int kIter = kPackK * (CW / 4) / 256;     // 16-byte loads per thread and chunk
  const int nt = b / pr.kt, kb = b % pr.kt;
  const int bn = pr.bn;
  const int64_t base = pr.b_row0 + (int64_t)b * PARTS * bn;
  const bool vec = aligned16(pr.B) && (pr.p & 3) == 0;
  for (int c0 = 0; c0 < bn; c0 += CW) {
    float4 vs[kIter];
#pragma unroll
    for (int it = 0; it < kIter; it++) {
      const int q = tid + it * 256;
      const int kk = q / (CW / 4), c4 = q % (CW / 4);
      const int64_t k = (int64_t)kb * kPackK + kk;
      const int64_t j = (int64_t)nt * bn + c0 + 4 * c4;
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
    for (int it = 0; it < kIter; it++) {
      const int q = tid + it * 256;
      const int kk = q / (CW / 4), c4 = q % (CW / 4);
      tile[kk][4 * c4 + 0] = vs[it].x;
      tile[kk][4 * c4 + 1] = vs[it].y;
      tile[kk][4 * c4 + 2] = vs[it].z;
      tile[kk][4 * c4 + 3] = vs[it].w;
    }
    __syncthreads();
    // column c = tid / 16 + 16 t of this chunk in round t: the 16 threads of
    // a half warp hold one column's 64 values
    constexpr int kCols = CW * kQuads / 256;
    uint32_t mxv[8];
#pragma unroll
    for (int t = 0; t < kCols; t++) {
      const int q = tid + t * 256;
      const int c = q / kQuads, kq = q % kQuads;
      const int64_t j = (int64_t)nt * bn + c0 + c;
      const int s = (MODE != kPackUnscaled && j < pr.p) ? scale_exponent(pr.tB[j]) : 0;
      const float4 x = make_float4(tile[4 * kq][c], tile[4 * kq + 1][c], tile[4 * kq + 2][c],
                                   tile[4 * kq + 3][c]);
      if (MODE == kPackUnscaled) mxv[t] = max4_bits(x);
      uint2 part[PARTS];
      split4<PARTS, MODE != kPackUnscaled>(x, s, part);
#pragma unroll
      for (int h = 0; h < PARTS; h++) pack[(base + h * bn + c0 + c) * kQuads + kq] = part[h];
    }
    if (MODE == kPackUnscaled) {
#pragma unroll
      for (int t = kCols; t < 8; t++) mxv[t] = 0;
      const uint32_t mx = half_warp_max8(mxv);
      const int t = (tid >> 1) & 7;
      const int64_t j = (int64_t)nt * bn + c0 + tid / kQuads + 16 * t;
      if ((tid & 1) == 0 && t < kCols && j < pr.p) pr.pB[(int64_t)kb * pr.p + j] = mx;
    }
    __syncthreads();
  }
}

// MODE: kPackUnscaled - no scaling; write the tile's row (A) / column (B)
//                       maxima to pA / pB; one block per pack tile;
//       kPackFix      - scale by 2^-s from the maxima in sA / tB; only the
//                       operands flagged by split_verify_kernel; a persistent
//                       grid over the pack tiles that returns at once when
//                       no operand of the table is flagged (*any == 0).
// Every thread first loads all its 16-byte vectors of a tile (eight of A, or
// four of a 64-column slice of B), then splits and stores them, so that each
// thread keeps several loads in flight.
template <int PARTS, int MODE>
__global__ void __launch_bounds__(256, 4)
split_pack_kernel(const SplitProb *__restrict__ probs, int nprobs, const int *__restrict__ map,
                  const int *__restrict__ flags, const int *__restrict__ any, int total_tiles,
                  uint2 *__restrict__ pack) {
  constexpr int kQuads = kPackK / 4;  // groups of four bf16 (8 bytes) per pack row
  constexpr int kAIter = kTcBM * kQuads / 256;
  static_assert(kAIter == 8, "eight A vectors per thread (one reduction slot each)");
  __shared__ float tile[kPackK][128 + 1];
  if (MODE == kPackFix && *any == 0) return;
  const int tid = threadIdx.x;
  for (int item = blockIdx.x; item < total_tiles; item += gridDim.x) {
    const int g =
        find_problem(probs, nprobs, map, item, [](const SplitProb &q) { return q.pack_start; });
    const SplitProb &pr = probs[g];
    const int local = item - pr.pack_start;
    const bool a_tile = local < pr.mt * pr.kt;
    if (MODE == kPackFix && !(flags[g] & (a_tile ? kFlagScaleA : kFlagScaleB))) continue;
    if (a_tile) {
      // A tile (mt, kb): rows mt*128.., k kb*64..; a warp covers two rows.
      const int mt = local / pr.kt, kb = local % pr.kt;
      const int64_t base = pr.a_row0 + (int64_t)local * PARTS * kTcBM;
      const bool vec = aligned16(pr.A) && (pr.m & 3) == 0;
      float4 xs[kAIter];
#pragma unroll
      for (int it = 0; it < kAIter; it++) {
        const int q = tid + it * 256;
        const int r = q / kQuads, kq = q % kQuads;
        const int64_t i = (int64_t)mt * kTcBM + r;
        const int64_t k = (int64_t)kb * kPackK + 4 * kq;
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
      if (MODE == kPackUnscaled) {
        // row r = tid / 16 + 16 it: the 16 threads of a half warp hold one
        // row's 64 values
        uint32_t mxv[8];
#pragma unroll
        for (int it = 0; it < 8; it++) mxv[it] = max4_bits(xs[it]);
        const uint32_t mx = half_warp_max8(mxv);
        const int t = (tid >> 1) & 7;
        const int64_t i = (int64_t)mt * kTcBM + tid / kQuads + 16 * t;
        if ((tid & 1) == 0 && i < pr.n) pr.pA[(int64_t)kb * pr.n + i] = mx;
      }
#pragma unroll
      for (int it = 0; it < kAIter; it++) {
        const int q = tid + it * 256;
        const int r = q / kQuads, kq = q % kQuads;
        const int64_t i = (int64_t)mt * kTcBM + r;
        const int s = (MODE != kPackUnscaled && i < pr.n) ? scale_exponent(pr.sA[i]) : 0;
        uint2 part[PARTS];
        split4<PARTS, MODE != kPackUnscaled>(xs[it], s, part);
#pragma unroll
        for (int h = 0; h < PARTS; h++) pack[(base + h * kTcBM + r) * kQuads + kq] = part[h];
      }
    } else {
      // B tile (nt, kb): columns nt*bn.., k kb*64..; transposed through shared
      // memory 128 columns at a time (64 for bn = 64) so both the read and the
      // write coalesce, with eight 16-byte loads per thread in flight.
      const int b = local - pr.mt * pr.kt;
      if (pr.bn % 128 == 0)
        pack_b_tile<PARTS, MODE, 128>(pr, b, pack, tile, tid);
      else
        pack_b_tile<PARTS, MODE, 64>(pr, b, pack, tile, tid);
    }
  }
}

// A row/column maximum outside [2^-40, 2^40] (or not finite) needs scaling;
// zero needs none.
__device__ __forceinline__ bool needs_scale(uint32_t max_bits) {
  return max_bits != 0 && (max_bits < 0x2B800000u /* 2^-40 */ || max_bits > 0x53800000u /* 2^40 */);
}

// Verify items of 32 rows/columns of one problem; WPI warps per item split
// its K blocks, 8 / WPI items per block (WPI from the table's longest K, so
// that short products do not pay for idle warps): the maximum of a row of A
// over its K blocks -> sA (columns of B -> tB), and flags[g] |= kFlagScaleA /
// kFlagScaleB (and *any) where a maximum is outside the range packed
// unscaled.
template <int WPI>
__global__ void __launch_bounds__(256)
split_verify_kernel(const SplitProb *__restrict__ probs, int nprobs, const int *__restrict__ map,
                    int total_items, int *__restrict__ flags, int *__restrict__ any,
                    bool write_cols) {
  __shared__ uint32_t part[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int sub = warp % WPI;
  const int item = blockIdx.x * (8 / WPI) + warp / WPI;
  const bool live = item < total_items;
  const SplitProb *pp = nullptr;
  int g = 0;
  int64_t w = 0;
  bool valid = false;
  uint32_t mx = 0;
  if (live) {
    g = find_problem(probs, nprobs, map, item, [](const SplitProb &q) { return q.ver_start; });
    pp = probs + g;
    w = (int64_t)(item - pp->ver_start) * 32 + lane;
    valid = w < (int64_t)pp->n + pp->p;
    if (valid) {
      const bool is_row = w < pp->n;
      const uint32_t *src = is_row ? pp->pA + w : pp->pB + (w - pp->n);
      const int64_t stride = is_row ? pp->n : pp->p;
#pragma unroll 4
      for (int kb = sub; kb < pp->kt; kb += WPI) mx = umax(mx, src[kb * stride]);
    }
  }
  if (WPI > 1) {
    part[warp][lane] = mx;
    __syncthreads();
    if (sub == 0)
#pragma unroll
      for (int q = 1; q < WPI; q++) mx = umax(mx, part[warp + q][lane]);
  }
  if (sub != 0 || !live) return;
  int bad = 0;
  if (valid) {
    const bool is_row = w < pp->n;
    if (is_row) pp->sA[w] = mx; else if (write_cols) pp->tB[w - pp->n] = mx;
    if (needs_scale(mx)) bad = is_row ? kFlagScaleA : kFlagScaleB;
  }
  const unsigned mask = __activemask();
  const unsigned a = __ballot_sync(mask, bad & kFlagScaleA);
  const unsigned b = __ballot_sync(mask, bad & kFlagScaleB);
  if (lane == 0 && (a || b)) {
    atomicOr(&flags[g], (a ? kFlagScaleA : 0) | (b ? kFlagScaleB : 0));
    atomicOr(any, 1);
  }
}

// One block per problem: writes the problem's index over its ranges of MMA
// tiles, pack tiles and scale-reduction items.
__global__ void __launch_bounds__(256)
split_maps_kernel(const SplitProb *__restrict__ probs, int *__restrict__ unit_map,
                  int *__restrict__ pack_map, int *__restrict__ ver_map) {
  const int g = blockIdx.x;
  const SplitProb &pr = probs[g];
  const int units = (int)split_units(pr);
  const int packs = pr.mt * pr.kt + pr.nt * pr.kt;
  if (unit_map)
    for (int i = threadIdx.x; i < units; i += blockDim.x) unit_map[pr.unit_start + i] = g;
  if (pack_map)
    for (int i = threadIdx.x; i < packs; i += blockDim.x) pack_map[pr.pack_start + i] = g;
  if (ver_map) {  // only tables that run split_verify_kernel
    const int vers = (int)verify_items(pr.n, pr.p);
    for (int i = threadIdx.x; i < vers; i += blockDim.x) ver_map[pr.ver_start + i] = g;
  }
}

}  // namespace

cudaError_t launch_split_maps(const SplitProb *d_probs, int nprobs, int *unit_map, int *pack_map,
                              int *ver_map, cudaStream_t s) {
  if (nprobs <= 0) return cudaSuccess;
  TraceScope ts("split_maps", s);
  split_maps_kernel<<<nprobs, 256, 0, s>>>(d_probs, unit_map, pack_map, ver_map);
  return cudaGetLastError();
}

cudaError_t launch_split_pack(TcKind kind, int mode, const SplitProb *d_probs, int nprobs,
                              int total_tiles, const int *map, const int *flags, const int *any,
                              void *pack_base, cudaStream_t s) {
  if (total_tiles <= 0) return cudaSuccess;
  TraceScope ts(mode == kPackFix ? "split_fix" : "split_pack", s);
  auto *pk = static_cast<uint2 *>(pack_base);
  const bool x6 = kind == kTcSplitBf16x6;
  // the fix pass: a persistent grid of one wave (4 blocks per SM, the launch
  // bound) over the tiles, so that its early return when nothing is flagged
  // costs a single wave of blocks
  const int grid = mode == kPackFix ? std::min(total_tiles, sm_count() * 4) : total_tiles;
#define MM_PACK(P, M) \
  split_pack_kernel<P, M><<<grid, 256, 0, s>>>(d_probs, nprobs, map, flags, any, total_tiles, pk)
  if (mode == kPackUnscaled) { if (x6) MM_PACK(3, kPackUnscaled); else MM_PACK(2, kPackUnscaled); }
  else { if (x6) MM_PACK(3, kPackFix); else MM_PACK(2, kPackFix); }
#undef MM_PACK
  return cudaGetLastError();
}

cudaError_t launch_split_verify(const SplitProb *d_probs, int nprobs, int64_t total_items,
                                const int *map, int *flags, int *any, int max_kt, cudaStream_t s,
                                bool write_cols) {
  if (nprobs <= 0 || total_items <= 0) return cudaSuccess;
  if (total_items > 0x7fffffffLL) return cudaErrorInvalidValue;
  TraceScope ts("split_verify", s);
  const int wpi = max_kt >= 64 ? 8 : (max_kt >= 32 ? 4 : (max_kt >= 16 ? 2 : 1));
  const int ti = (int)total_items;
  const unsigned blocks = (unsigned)((total_items * wpi + 7) / 8);
#define MM_VERIFY(W) \
  split_verify_kernel<W><<<blocks, 256, 0, s>>>(d_probs, nprobs, map, ti, flags, any, write_cols)
  if (wpi == 8) MM_VERIFY(8);
  else if (wpi == 4) MM_VERIFY(4);
  else if (wpi == 2) MM_VERIFY(2);
  else MM_VERIFY(1);
#undef MM_VERIFY
  return cudaGetLastError();
}

}  // namespace mm
