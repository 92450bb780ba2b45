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
__device__ __forceinline__ uint32_t to_e4m3x4(float x0, float x1, float x2, float x3, int e) {
  const __nv_fp8x2_storage_t lo =
      __nv_cvt_float2_to_fp8x2(make_float2(ldexpf(x0, -e), ldexpf(x1, -e)), __NV_SATFINITE, __NV_E4M3);
  const __nv_fp8x2_storage_t hi =
      __nv_cvt_float2_to_fp8x2(make_float2(ldexpf(x2, -e), ldexpf(x3, -e)), __NV_SATFINITE, __NV_E4M3);
  return (uint32_t)lo | ((uint32_t)hi << 16);
}

__global__ void __launch_bounds__(256)
fp8_pack_kernel(const SplitProb *__restrict__ probs, int nprobs, const int *__restrict__ map,
                uint32_t *__restrict__ pack) {
  const int item = blockIdx.x;
  const int g =
      find_problem(probs, nprobs, map, item, [](const SplitProb &q) { return q.pack_start; });
  const SplitProb &pr = probs[g];
  const int local = item - pr.pack_start;
  const int tid = threadIdx.x;
  constexpr int kQuads = kK / 4;  // 32-bit words per pack row
  if (local < pr.mt * pr.kt) {
    // A tile (mt, kb): 128 rows x 128 k; a warp writes one 128-byte row.
    const int mt = local / pr.kt, kb = local % pr.kt;
    const int64_t base = pr.a_row0 + (int64_t)local * kTcBM;
    for (int q = tid; q < kTcBM * kQuads; q += 256) {
      const int r = q / kQuads, kq = q % kQuads;
      const int64_t i = (int64_t)mt * kTcBM + r;
      const int64_t k = (int64_t)kb * kK + 4 * kq;
      float x[4] = {0.f, 0.f, 0.f, 0.f};
      int e = 0;
      if (i < pr.n) {
        const float *row = pr.A + i * pr.m;
#pragma unroll
        for (int t = 0; t < 4; t++)
          if (k + t < pr.m) x[t] = row[k + t];
        e = e4m3_exponent(pr.sA[i]);
      }
      pack[(base + r) * kQuads + kq] = to_e4m3x4(x[0], x[1], x[2], x[3], e);
    }
  } else {
    // B tile (nt, kb): bn columns x 128 k, transposed through shared memory
    // 32 columns at a time.
    __shared__ float tile[kK][32 + 1];
    const int b = local - pr.mt * pr.kt;
    const int nt = b / pr.kt, kb = b % pr.kt;
    const int bn = pr.bn;
    const int64_t base = pr.b_row0 + (int64_t)b * bn;
    for (int c0 = 0; c0 < bn; c0 += 32) {
      for (int q = tid; q < kK * 32; q += 256) {
        const int kk = q / 32, c = q % 32;
        const int64_t k = (int64_t)kb * kK + kk;
        const int64_t j = (int64_t)nt * bn + c0 + c;
        tile[kk][c] = (k < pr.m && j < pr.p) ? pr.B[k * pr.p + j] : 0.f;
      }
      __syncthreads();
      for (int q = tid; q < 32 * kQuads; q += 256) {
        const int c = q / kQuads, kq = q % kQuads;
        const int64_t j = (int64_t)nt * bn + c0 + c;
        const int e = j < pr.p ? e4m3_exponent(pr.tB[j]) : 0;
        pack[(base + c0 + c) * kQuads + kq] =
            to_e4m3x4(tile[4 * kq][c], tile[4 * kq + 1][c], tile[4 * kq + 2][c],
                      tile[4 * kq + 3][c], e);
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
