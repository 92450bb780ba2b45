// FP8 (e4m3) path: operand conversion for the e4m3 kind of the tensor-core
// kernel (tc_gemm.cu).
//
// Every row of A and column of B is scaled by a power of two 2^-e chosen from
// its largest magnitude so that the largest scaled entry lies in [128, 256)
// (below the e4m3 maximum 448), then rounded to e4m3 (round to nearest even,
// saturating).  The tensor cores multiply the e4m3 operands with FP32
// accumulation and the epilogue multiplies by 2^(e_i + e_j) exactly.  With
// three significand bits the result is a low-precision estimate: its error
// against the FP64 oracle is measured and reported, not bounded.  Not in the
// paper.
#include <cuda_fp8.h>

#include "split_common.cuh"

namespace mm {
namespace {

constexpr int kK = 128;  // e4m3 values per pack row (128 bytes)

__device__ __forceinline__ int e4m3_exponent(uint32_t max_bits) {
  const float f = __uint_as_float(max_bits);
  return (f > 0.0f && f <= 3.402823466e38f) ? scale_exponent(max_bits) - 7 : 0;
}

// Four consecutive values scaled by 2^-e -> four e4m3 bytes (first in the
// lowest byte).
__device__ __forceinline__ uint32_t to_e4m3x4(float4 x, int e) {
  const __nv_fp8x2_storage_t lo = __nv_cvt_float2_to_fp8x2(
      make_float2(scale_pow2(x.x, -e), scale_pow2(x.y, -e)), __NV_SATFINITE, __NV_E4M3);
  const __nv_fp8x2_storage_t hi = __nv_cvt_float2_to_fp8x2(
      make_float2(scale_pow2(x.z, -e), scale_pow2(x.w, -e)), __NV_SATFINITE, __NV_E4M3);
  return (uint32_t)lo | ((uint32_t)hi << 16);
}

__device__ __forceinline__ bool aligned16(const void *p) {
  return (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
}

// One block per pack tile.  A tile (mt, kb): 128 rows x 128 k, read as
// 16-byte vectors (eight per thread in flight), written as one 128-byte pack
// row per row.  B tile (nt, kb): bn columns x 128 k, transposed through
// shared memory 64 columns at a time (eight 16-byte loads per thread in
// flight), written as one pack row per column, 16 bytes per store.
__global__ void __launch_bounds__(256, 4)
fp8_pack_kernel(const SplitProb *__restrict__ probs, int nprobs, const int *__restrict__ map,
                uint32_t *__restrict__ pack) {
  constexpr int kQuads = kK / 4;            // 32-bit words per pack row
  constexpr int kBatch = 8;                 // vectors per thread in flight
  __shared__ float tile[kK][64 + 1];
  const int item = blockIdx.x;
  const int g =
      find_problem(probs, nprobs, map, item, [](const SplitProb &q) { return q.pack_start; });
  const SplitProb &pr = probs[g];
  const int local = item - pr.pack_start;
  const int tid = threadIdx.x;
  if (local < pr.mt * pr.kt) {
    const int mt = local / pr.kt, kb = local % pr.kt;
    const int64_t base = pr.a_row0 + (int64_t)local * kTcBM;
    const bool vec = aligned16(pr.A) && (pr.m & 3) == 0;
    for (int q0 = 0; q0 < kTcBM * kQuads; q0 += 256 * kBatch) {
      float4 xs[kBatch];
#pragma unroll
      for (int it = 0; it < kBatch; it++) {
        const int q = q0 + tid + it * 256;
        const int r = q / kQuads, kq = q % kQuads;
        const int64_t i = (int64_t)mt * kTcBM + r;
        const int64_t k = (int64_t)kb * kK + 4 * kq;
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
      for (int it = 0; it < kBatch; it++) {
        const int q = q0 + tid + it * 256;
        const int r = q / kQuads, kq = q % kQuads;
        const int64_t i = (int64_t)mt * kTcBM + r;
        const int e = i < pr.n ? e4m3_exponent(pr.sA[i]) : 0;
        pack[(base + r) * kQuads + kq] = to_e4m3x4(xs[it], e);
      }
    }
  } else {
    const int b = local - pr.mt * pr.kt;
    const int nt = b / pr.kt, kb = b % pr.kt;
    const int bn = pr.bn;
    const int64_t base = pr.b_row0 + (int64_t)b * bn;
    const bool vec = aligned16(pr.B) && (pr.p & 3) == 0;
    for (int c0 = 0; c0 < bn; c0 += 64) {
      float4 vs[kBatch];
#pragma unroll
      for (int it = 0; it < kBatch; it++) {
        const int q = tid + it * 256;  // 128 k rows x 16 vectors of 4 columns
        const int kk = q / 16, c4 = q % 16;
        const int64_t k = (int64_t)kb * kK + kk;
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
      for (int it = 0; it < kBatch; it++) {
        const int q = tid + it * 256;
        const int kk = q / 16, c4 = q % 16;
        tile[kk][4 * c4 + 0] = vs[it].x;
        tile[kk][4 * c4 + 1] = vs[it].y;
        tile[kk][4 * c4 + 2] = vs[it].z;
        tile[kk][4 * c4 + 3] = vs[it].w;
      }
      __syncthreads();
      // a lane per column (the warp reads 32 consecutive columns of a tile
      // row: no bank conflicts), 16 k values per item written as 16 bytes
      for (int q = tid; q < 64 * (kK / 16); q += 256) {
        const int c = q % 64, k16 = q / 64;
        const int64_t j = (int64_t)nt * bn + c0 + c;
        const int e = j < pr.p ? e4m3_exponent(pr.tB[j]) : 0;
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

}  // namespace

cudaError_t launch_fp8_pack(const SplitProb *d_probs, int nprobs, int total_tiles, const int *map,
                            void *pack_base, cudaStream_t s) {
  if (total_tiles <= 0) return cudaSuccess;
  TraceScope ts("fp8_pack", s);
  fp8_pack_kernel<<<total_tiles, 256, 0, s>>>(d_probs, nprobs, map,
                                              static_cast<uint32_t *>(pack_base));
  return cudaGetLastError();
}

}  // namespace mm
