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
//                       orders like the value for non-negative floats).
//   split_pack_kernel   one block per 128 x 64 tile of A or bn x 64 tile of
//                       B^T: scale, split, write the bf16 parts (hi, lo - or
//                       hi, mid, lo for the three-part split) of the pack
//                       (layout in mm_internal.h); zero outside the matrix
//                       so the tensor-core kernel needs no edge checks.
#include "split_common.cuh"

namespace mm {
namespace {

constexpr int kRowsPerScaleItem = 8;    // warps per block, one row each
constexpr int kColStrip = 32;
constexpr int kRowChunk = 256;

__global__ void __launch_bounds__(256)
split_scale_kernel(const SplitProb *__restrict__ probs, int nprobs) {
  const int item = blockIdx.x;
  const int g = find_problem(probs, nprobs, item, [](const SplitProb &q) { return q.red_start; });
  const SplitProb &pr = probs[g];
  const int local = item - pr.red_start;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (local < pr.red_a) {
    const int64_t i = (int64_t)local * kRowsPerScaleItem + warp;
    if (i >= pr.n) return;
    const float *row = pr.A + i * pr.m;
    uint32_t mx = 0;
    for (int64_t k = lane; k < pr.m; k += 32) {
      const uint32_t b = __float_as_uint(row[k]) & 0x7fffffffu;
      mx = b > mx ? b : mx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const uint32_t t = __shfl_xor_sync(0xffffffffu, mx, o);
      mx = t > mx ? t : mx;
    }
    if (lane == 0) pr.sA[i] = mx;
  } else {
    __shared__ uint32_t part[8][kColStrip];
    const int b = local - pr.red_a;
    const int strips = (pr.p + kColStrip - 1) / kColStrip;
    const int strip = b % strips, chunk = b / strips;
    const int64_t col = (int64_t)strip * kColStrip + lane;
    const int64_t r0 = (int64_t)chunk * kRowChunk + warp * (kRowChunk / 8);
    uint32_t mx = 0;
    if (col < pr.p) {
#pragma unroll 8
      for (int r = 0; r < kRowChunk / 8; r++) {
        const int64_t k = r0 + r;
        if (k < pr.m) {
          const uint32_t v = __float_as_uint(pr.B[k * pr.p + col]) & 0x7fffffffu;
          mx = v > mx ? v : mx;
        }
      }
    }
    part[warp][lane] = mx;
    __syncthreads();
    if (warp == 0) {
#pragma unroll
      for (int w = 1; w < 8; w++) mx = part[w][lane] > mx ? part[w][lane] : mx;
      if (col < pr.p) atomicMax(&pr.tB[col], mx);
    }
  }
}

// Splits two values scaled by 2^-s into PARTS bf16 pairs: part 0 = RN(y),
// part q = RN(y - part 0 - ... - part q-1).  Every remainder is exact in FP32
// (the difference of a float and its rounding to fewer bits), so
// y = sum of parts + d with |d| <= 2^(-8*PARTS) |y|.
template <int PARTS>
__device__ __forceinline__ void split_pair(float x0, float x1, int s, __nv_bfloat162 (&out)[PARTS]) {
  float y0 = ldexpf(x0, -s), y1 = ldexpf(x1, -s);
#pragma unroll
  for (int q = 0; q < PARTS; q++) {
    out[q] = __floats2bfloat162_rn(y0, y1);
    const float2 h = __bfloat1622float2(out[q]);
    y0 -= h.x;
    y1 -= h.y;
  }
}

template <int PARTS>
__global__ void __launch_bounds__(256)
split_pack_kernel(const SplitProb *__restrict__ probs, int nprobs,
                  __nv_bfloat162 *__restrict__ pack) {
  const int item = blockIdx.x;
  const int g = find_problem(probs, nprobs, item, [](const SplitProb &q) { return q.pack_start; });
  const SplitProb &pr = probs[g];
  const int local = item - pr.pack_start;
  const int tid = threadIdx.x;
  constexpr int kPairs = kPackK / 2;  // bf16x2 per pack row
  if (local < pr.mt * pr.kt) {
    // A tile (mt, kb): rows mt*128.., k kb*64..; a warp covers one row.
    const int mt = local / pr.kt, kb = local % pr.kt;
    const int64_t base = pr.a_row0 + (int64_t)local * PARTS * kTcBM;
    for (int q = tid; q < kTcBM * kPairs; q += 256) {
      const int r = q / kPairs, kp = q % kPairs;
      const int64_t i = (int64_t)mt * kTcBM + r;
      const int64_t k = (int64_t)kb * kPackK + 2 * kp;
      float x0 = 0.f, x1 = 0.f;
      int s = 0;
      if (i < pr.n) {
        const float *row = pr.A + i * pr.m;
        if (k < pr.m) x0 = row[k];
        if (k + 1 < pr.m) x1 = row[k + 1];
        s = scale_exponent(pr.sA[i]);
      }
      __nv_bfloat162 part[PARTS];
      split_pair<PARTS>(x0, x1, s, part);
#pragma unroll
      for (int h = 0; h < PARTS; h++) pack[(base + h * kTcBM + r) * kPairs + kp] = part[h];
    }
  } else {
    // B tile (nt, kb): columns nt*bn.., k kb*64..; transposed through shared
    // memory 64 columns at a time so both the read and the write coalesce.
    __shared__ float tile[kPackK][64 + 1];
    const int b = local - pr.mt * pr.kt;
    const int nt = b / pr.kt, kb = b % pr.kt;
    const int bn = pr.bn;
    const int64_t base = pr.b_row0 + (int64_t)b * PARTS * bn;
    for (int c0 = 0; c0 < bn; c0 += 64) {
      for (int q = tid; q < kPackK * 64; q += 256) {
        const int kk = q / 64, c = q % 64;
        const int64_t k = (int64_t)kb * kPackK + kk;
        const int64_t j = (int64_t)nt * bn + c0 + c;
        tile[kk][c] = (k < pr.m && j < pr.p) ? pr.B[k * pr.p + j] : 0.f;
      }
      __syncthreads();
      for (int q = tid; q < 64 * kPairs; q += 256) {
        const int c = q / kPairs, kp = q % kPairs;
        const int64_t j = (int64_t)nt * bn + c0 + c;
        const int s = j < pr.p ? scale_exponent(pr.tB[j]) : 0;
        __nv_bfloat162 part[PARTS];
        split_pair<PARTS>(tile[2 * kp][c], tile[2 * kp + 1][c], s, part);
#pragma unroll
        for (int h = 0; h < PARTS; h++) pack[(base + h * bn + c0 + c) * kPairs + kp] = part[h];
      }
      __syncthreads();
    }
  }
}

}  // namespace

cudaError_t launch_split_scale(const SplitProb *d_probs, int nprobs, int total_items,
                               cudaStream_t s) {
  if (total_items <= 0) return cudaSuccess;
  TraceScope ts("split_scale", s);
  split_scale_kernel<<<total_items, 256, 0, s>>>(d_probs, nprobs);
  return cudaGetLastError();
}

cudaError_t launch_split_pack(TcKind kind, const SplitProb *d_probs, int nprobs, int total_tiles,
                              void *pack_base, cudaStream_t s) {
  if (total_tiles <= 0) return cudaSuccess;
  TraceScope ts("split_pack", s);
  auto *pk = static_cast<__nv_bfloat162 *>(pack_base);
  if (kind == kTcSplitBf16x6)
    split_pack_kernel<3><<<total_tiles, 256, 0, s>>>(d_probs, nprobs, pk);
  else
    split_pack_kernel<2><<<total_tiles, 256, 0, s>>>(d_probs, nprobs, pk);
  return cudaGetLastError();
}

}  // namespace mm
