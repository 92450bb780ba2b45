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
//   split_scale_kernel  max |a_ir| per row of A (a warp per row) and
//                       max |b_rj| per column of B (strips of 32 columns x
//                       256 rows, atomicMax on the float bit pattern, which
//                       orders like the value for non-negative floats); used
//                       by the e4m3 path, whose conversion needs the scales
//                       first.
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
#include "split_common.cuh"

namespace mm {
namespace {

constexpr int kRowsPerScaleItem = 8;    // warps per block, one row each
constexpr int kColStrip = 32;
constexpr int kRowChunk = 256;

__device__ __forceinline__ uint32_t abs_bits(float x) { return __float_as_uint(x) & 0x7fffffffu; }

__device__ __forceinline__ uint32_t umax(uint32_t a, uint32_t b) { return a > b ? a : b; }

__device__ __forceinline__ bool aligned16(const void *p) {
  return (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
}

__global__ void __launch_bounds__(256)
split_scale_kernel(const SplitProb *__restrict__ probs, int nprobs, const int *__restrict__ map) {
  const int item = blockIdx.x;
  const int g =
      find_problem(probs, nprobs, map, item, [](const SplitProb &q) { return q.red_start; });
  const SplitProb &pr = probs[g];
  const int local = item - pr.red_start;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (local < pr.red_a) {
    // a warp per row of A; 16-byte loads when every row start is aligned
    const int64_t i = (int64_t)local * kRowsPerScaleItem + warp;
    if (i >= pr.n) return;
    const float *row = pr.A + i * pr.m;
    uint32_t mx = 0;
    if (aligned16(pr.A) && (pr.m & 3) == 0) {
      const float4 *r4 = reinterpret_cast<const float4 *>(row);
      const int64_t m4 = pr.m >> 2;
#pragma unroll 4
      for (int64_t k = lane; k < m4; k += 32) {
        const float4 v = r4[k];
        mx = umax(mx, umax(umax(abs_bits(v.x), abs_bits(v.y)), umax(abs_bits(v.z), abs_bits(v.w))));
      }
    } else {
#pragma unroll 4
      for (int64_t k = lane; k < pr.m; k += 32) mx = umax(mx, abs_bits(row[k]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = umax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) pr.sA[i] = mx;
  } else {
    // a strip of 32 columns x 256 rows of B; the block's maxima are merged
    // into the column words with atomicMax
    __shared__ uint32_t part[32][kColStrip + 1];
    const int b = local - pr.red_a;
    const int strips = (pr.p + kColStrip - 1) / kColStrip;
    const int strip = b % strips, chunk = b / strips;
    const int64_t c0 = (int64_t)strip * kColStrip;
    const int64_t r0 = (int64_t)chunk * kRowChunk;
    const int tid = threadIdx.x;
    if (aligned16(pr.B) && (pr.p & 3) == 0 && c0 + kColStrip <= pr.p) {
      // 8 threads x 4 columns cover a 128-byte row segment; 32 row groups
      const int cq = tid & 7, grp = tid >> 3;
      uint32_t m0 = 0, m1 = 0, m2 = 0, m3 = 0;
#pragma unroll 4
      for (int r = grp; r < kRowChunk; r += 32) {
        const int64_t k = r0 + r;
        if (k < pr.m) {
          const float4 v = *reinterpret_cast<const float4 *>(pr.B + k * pr.p + c0 + 4 * cq);
          m0 = umax(m0, abs_bits(v.x));
          m1 = umax(m1, abs_bits(v.y));
          m2 = umax(m2, abs_bits(v.z));
          m3 = umax(m3, abs_bits(v.w));
        }
      }
      part[grp][4 * cq + 0] = m0;
      part[grp][4 * cq + 1] = m1;
      part[grp][4 * cq + 2] = m2;
      part[grp][4 * cq + 3] = m3;
      __syncthreads();
      if (warp == 0) {
        uint32_t mx = 0;
#pragma unroll 8
        for (int w = 0; w < 32; w++) mx = umax(mx, part[w][lane]);
        atomicMax(&pr.tB[c0 + lane], mx);
      }
    } else {
      const int64_t col = c0 + lane;
      uint32_t mx = 0;
      if (col < pr.p) {
#pragma unroll 8
        for (int r = warp; r < kRowChunk; r += 8) {
          const int64_t k = r0 + r;
          if (k < pr.m) mx = umax(mx, abs_bits(pr.B[k * pr.p + col]));
        }
      }
      part[warp][lane] = mx;
      __syncthreads();
      if (warp == 0) {
#pragma unroll
        for (int w = 1; w < 8; w++) mx = umax(mx, part[w][lane]);
        if (col < pr.p) atomicMax(&pr.tB[col], mx);
      }
    }
  }
}

// Splits four values scaled by 2^-s into PARTS groups of four bf16 (two
// bf16x2 words each): part 0 = RN(y), part q = RN(y - part 0 - ... - part
// q-1).  Every remainder is exact in FP32 (the difference of a float and its
// rounding to fewer bits), so y = sum of parts + d, |d| <= 2^(-8*PARTS) |y|.
template <int PARTS>
__device__ __forceinline__ void split4(float4 x, int s, uint2 (&out)[PARTS]) {
  float y[4] = {ldexpf(x.x, -s), ldexpf(x.y, -s), ldexpf(x.z, -s), ldexpf(x.w, -s)};
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

// max over the 16 lanes of a half warp (lanes 0-15 or 16-31)
__device__ __forceinline__ uint32_t half_warp_max(uint32_t v) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v = umax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// MODE: kPackUnscaled - no scaling; write the tile's row (A) / column (B)
//                       maxima to pA / pB;
//       kPackFix      - scale by 2^-s from the maxima in sA / tB; only the
//                       operands flagged by split_verify_kernel (the other
//                       blocks return).
template <int PARTS, int MODE>
__global__ void __launch_bounds__(256)
split_pack_kernel(const SplitProb *__restrict__ probs, int nprobs, const int *__restrict__ map,
                  const int *__restrict__ flags, uint2 *__restrict__ pack) {
  const int item = blockIdx.x;
  const int g =
      find_problem(probs, nprobs, map, item, [](const SplitProb &q) { return q.pack_start; });
  const SplitProb &pr = probs[g];
  const int local = item - pr.pack_start;
  const int tid = threadIdx.x;
  constexpr int kQuads = kPackK / 4;  // groups of four bf16 (8 bytes) per pack row
  const bool a_tile = local < pr.mt * pr.kt;
  if (MODE == kPackFix && !(flags[g] & (a_tile ? kFlagScaleA : kFlagScaleB))) return;
  if (a_tile) {
    // A tile (mt, kb): rows mt*128.., k kb*64..; a warp covers two rows.
    const int mt = local / pr.kt, kb = local % pr.kt;
    const int64_t base = pr.a_row0 + (int64_t)local * PARTS * kTcBM;
    const bool vec = aligned16(pr.A) && (pr.m & 3) == 0;
    for (int q = tid; q < kTcBM * kQuads; q += 256) {
      const int r = q / kQuads, kq = q % kQuads;
      const int64_t i = (int64_t)mt * kTcBM + r;
      const int64_t k = (int64_t)kb * kPackK + 4 * kq;
      float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
      int s = 0;
      if (i < pr.n) {
        const float *row = pr.A + i * pr.m;
        if (vec && k + 4 <= pr.m) {
          x = *reinterpret_cast<const float4 *>(row + k);
        } else {
          if (k < pr.m) x.x = row[k];
          if (k + 1 < pr.m) x.y = row[k + 1];
          if (k + 2 < pr.m) x.z = row[k + 2];
          if (k + 3 < pr.m) x.w = row[k + 3];
        }
        if (MODE != kPackUnscaled) s = scale_exponent(pr.sA[i]);
      }
      if (MODE == kPackUnscaled) {
        // the 16 threads of a half warp hold one row's 64 values
        const uint32_t mx = half_warp_max(max4_bits(x));
        if (kq == 0 && i < pr.n) pr.pA[(int64_t)kb * pr.n + i] = mx;
      }
      uint2 part[PARTS];
      split4<PARTS>(x, s, part);
#pragma unroll
      for (int h = 0; h < PARTS; h++) pack[(base + h * kTcBM + r) * kQuads + kq] = part[h];
    }
  } else {
    // B tile (nt, kb): columns nt*bn.., k kb*64..; transposed through shared
    // memory 64 columns at a time so both the read and the write coalesce.
    __shared__ float tile[kPackK][64 + 1];
    const int b = local - pr.mt * pr.kt;
    const int nt = b / pr.kt, kb = b % pr.kt;
    const int bn = pr.bn;
    const int64_t base = pr.b_row0 + (int64_t)b * PARTS * bn;
    const bool vec = aligned16(pr.B) && (pr.p & 3) == 0;
    for (int c0 = 0; c0 < bn; c0 += 64) {
      for (int q = tid; q < kPackK * 16; q += 256) {
        const int kk = q / 16, c4 = q % 16;
        const int64_t k = (int64_t)kb * kPackK + kk;
        const int64_t j = (int64_t)nt * bn + c0 + 4 * c4;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (k < pr.m) {
          const float *src = pr.B + k * pr.p + j;
          if (vec && j + 4 <= pr.p) {
            v = *reinterpret_cast<const float4 *>(src);
          } else {
            if (j < pr.p) v.x = src[0];
            if (j + 1 < pr.p) v.y = src[1];
            if (j + 2 < pr.p) v.z = src[2];
            if (j + 3 < pr.p) v.w = src[3];
          }
        }
        tile[kk][4 * c4 + 0] = v.x;
        tile[kk][4 * c4 + 1] = v.y;
        tile[kk][4 * c4 + 2] = v.z;
        tile[kk][4 * c4 + 3] = v.w;
      }
      __syncthreads();
      for (int q = tid; q < 64 * kQuads; q += 256) {
        const int c = q / kQuads, kq = q % kQuads;
        const int64_t j = (int64_t)nt * bn + c0 + c;
        const int s = (MODE != kPackUnscaled && j < pr.p) ? scale_exponent(pr.tB[j]) : 0;
        const float4 x = make_float4(tile[4 * kq][c], tile[4 * kq + 1][c], tile[4 * kq + 2][c],
                                     tile[4 * kq + 3][c]);
        if (MODE == kPackUnscaled) {
          // the 16 threads of a half warp hold one column's 64 values
          const uint32_t mx = half_warp_max(max4_bits(x));
          if (kq == 0 && j < pr.p) pr.pB[(int64_t)kb * pr.p + j] = mx;
        }
        uint2 part[PARTS];
        split4<PARTS>(x, s, part);
#pragma unroll
        for (int h = 0; h < PARTS; h++) pack[(base + h * bn + c0 + c) * kQuads + kq] = part[h];
      }
      __syncthreads();
    }
  }
}

// A row/column maximum outside [2^-40, 2^40] (or not finite) needs scaling;
// zero needs none.
__device__ __forceinline__ bool needs_scale(uint32_t max_bits) {
  return max_bits != 0 && (max_bits < 0x2B800000u /* 2^-40 */ || max_bits > 0x53800000u /* 2^40 */);
}

// Blocks (x: 32 rows/columns, y: problems; 8 warps split the K blocks): the
// maximum of a row of A over its K blocks -> sA (columns of B -> tB), and
// flags[g] |= kFlagScaleA / kFlagScaleB where a maximum is outside the range
// packed unscaled.
__global__ void __launch_bounds__(256)
split_verify_kernel(const SplitProb *__restrict__ probs, int nprobs, int *__restrict__ flags,
                    bool write_cols) {
  __shared__ uint32_t part[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int g = blockIdx.y; g < nprobs; g += gridDim.y) {
    const SplitProb &pr = probs[g];
    const int64_t w = (int64_t)blockIdx.x * 32 + lane;
    const bool is_row = w < pr.n;
    const bool valid = w < (int64_t)pr.n + pr.p;
    const uint32_t *src = is_row ? pr.pA + w : pr.pB + (w - pr.n);
    const int64_t stride = is_row ? pr.n : pr.p;
    uint32_t mx = 0;
    if (valid) {
#pragma unroll 4
      for (int kb = warp; kb < pr.kt; kb += 8) mx = umax(mx, src[kb * stride]);
    }
    part[warp][lane] = mx;
    __syncthreads();
    int bad = 0;
    if (warp == 0 && valid) {
#pragma unroll
      for (int q = 1; q < 8; q++) mx = umax(mx, part[q][lane]);
      if (is_row) pr.sA[w] = mx; else if (write_cols) pr.tB[w - pr.n] = mx;
      if (needs_scale(mx)) bad = is_row ? kFlagScaleA : kFlagScaleB;
    }
    const int any = __syncthreads_or(bad);
    if (any) {
      const int a = __syncthreads_or(bad & kFlagScaleA);
      const int b = __syncthreads_or(bad & kFlagScaleB);
      if (threadIdx.x == 0) atomicOr(&flags[g], (a ? kFlagScaleA : 0) | (b ? kFlagScaleB : 0));
    }
  }
}

// One block per problem: writes the problem's index over its ranges of MMA
// tiles, pack tiles and scale-reduction items.
__global__ void __launch_bounds__(256)
split_maps_kernel(const SplitProb *__restrict__ probs, int *__restrict__ unit_map,
                  int *__restrict__ pack_map, int *__restrict__ red_map) {
  const int g = blockIdx.x;
  const SplitProb &pr = probs[g];
  const int units = (int)split_units(pr);
  const int packs = pr.mt * pr.kt + pr.nt * pr.kt;
  const int reds = pr.red_a + ((pr.p + kColStrip - 1) / kColStrip) *
                                  ((pr.m + kRowChunk - 1) / kRowChunk);
  for (int i = threadIdx.x; i < units; i += blockDim.x) unit_map[pr.unit_start + i] = g;
  for (int i = threadIdx.x; i < packs; i += blockDim.x) pack_map[pr.pack_start + i] = g;
  if (red_map)  // only tables that run split_scale_kernel (the e4m3 path)
    for (int i = threadIdx.x; i < reds; i += blockDim.x) red_map[pr.red_start + i] = g;
}

}  // namespace

cudaError_t launch_split_maps(const SplitProb *d_probs, int nprobs, int *unit_map, int *pack_map,
                              int *red_map, cudaStream_t s) {
  if (nprobs <= 0) return cudaSuccess;
  TraceScope ts("split_maps", s);
  split_maps_kernel<<<nprobs, 256, 0, s>>>(d_probs, unit_map, pack_map, red_map);
  return cudaGetLastError();
}

cudaError_t launch_split_scale(const SplitProb *d_probs, int nprobs, int total_items,
                               const int *map, cudaStream_t s) {
  if (total_items <= 0) return cudaSuccess;
  TraceScope ts("split_scale", s);
  split_scale_kernel<<<total_items, 256, 0, s>>>(d_probs, nprobs, map);
  return cudaGetLastError();
}

cudaError_t launch_split_pack(TcKind kind, int mode, const SplitProb *d_probs, int nprobs,
                              int total_tiles, const int *map, const int *flags, void *pack_base,
                              cudaStream_t s) {
  if (total_tiles <= 0) return cudaSuccess;
  TraceScope ts(mode == kPackFix ? "split_fix" : "split_pack", s);
  auto *pk = static_cast<uint2 *>(pack_base);
  const bool x6 = kind == kTcSplitBf16x6;
#define MM_PACK(P, M) split_pack_kernel<P, M><<<total_tiles, 256, 0, s>>>(d_probs, nprobs, map, flags, pk)
  if (mode == kPackUnscaled) { if (x6) MM_PACK(3, kPackUnscaled); else MM_PACK(2, kPackUnscaled); }
  else { if (x6) MM_PACK(3, kPackFix); else MM_PACK(2, kPackFix); }
#undef MM_PACK
  return cudaGetLastError();
}

cudaError_t launch_split_verify(const SplitProb *d_probs, int nprobs, int64_t max_words,
                                int *flags, cudaStream_t s, bool write_cols) {
  if (nprobs <= 0 || max_words <= 0) return cudaSuccess;
  TraceScope ts("split_verify", s);
  dim3 grid((unsigned)((max_words + 31) / 32), (unsigned)(nprobs < 65535 ? nprobs : 65535));
  split_verify_kernel<<<grid, 256, 0, s>>>(d_probs, nprobs, flags, write_cols);
  return cudaGetLastError();
}

}  // namespace mm
