// FP64 product C = A.B emulated on the e4m3 tensor cores (Ozaki scheme).
//
// Method: K. Ozaki, T. Ogita, S. Oishi, S. M. Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applicability", Numer. Algorithms 59 (2012): split
// every operand into slices whose pairwise products a low-precision matrix
// unit computes without rounding, then add the slice products in the working
// precision.  This library's variant (not in the paper, whose double-precision
// kernels use FP64 arithmetic directly):
//
//   * Row i of A is scaled by 2^-sigma_i, sigma_i = ilogb(max_r |a_ir|) + 2,
//     so |a_ir| 2^-sigma_i < 1/2; column j of B by 2^-tau_j likewise.  The
//     scaled magnitude, truncated to 5S fraction bits, is the integer
//     F = floor(|a| 2^(5S - sigma)) < 2^(5S - 1) (S <= 12: 59 bits), written
//     in balanced base 32: G = F + 16 (32^S - 1) / 31 (16 added to every
//     base-32 position), then d_t = g_t - 16 with g_t = (G >> 5(S-1-t)) & 31
//     for t >= 1 and g_0 = G >> 5(S-1) unmasked, so d_t lies in [-16, 15]
//     (t >= 1), d_0 in [0, 16], and sum_t d_t 32^(S-1-t) = F.  With the sign
//     of a on every digit:
//         a 2^-sigma = sum_t d_t 32^-(t+1) + delta,  |delta| < 2^(-5S).
//     Every digit (|d| <= 16) is exact in e4m3; five bits per slice instead
//     of four cut the slices (and the S(S+1)/2 level products) for the same
//     precision.
//   * Level L = 0..S-1 collects the slice products of equal weight:
//         D_L = sum_{t+u=L} A_t B_u,
//     one tensor-core product along a K of (L+1) slices: A's slices 0..L
//     against B's slices L..0.  Each term is at most 256, a level at most
//     256 S mc, so with K cut into chunks of mc <= (2^24 - 1) / (256 S)
//     columns (a multiple of 128) every D_L is an integer below 2^24 and
//     FP32 accumulation (and the tail split's FP32 partial sums) is exact.
//     Pairs with t + u >= S are dropped.
//   * c_ij = 2^(sigma_i + tau_j) * sum_L 32^-(L+2) D_L[i][j] (summed over
//     the chunks too), formed exactly in 128-bit integers and rounded once
//     to FP64: the double nearest to the kept digit products.
//
// Error: a term a_ir b_rj loses at most (S + 2) 2^(sigma_i + tau_j - 5S - 1)
// (both truncations and the dropped pairs), and zero entries lose nothing,
// so |c^_ij - c_ij| <= (S + 2) 2^(sigma_i + tau_j - 5S - 1) #{r : a_ir b_rj != 0}
// plus the final rounding (half an ulp of c^_ij).  Relative to (|A||B|)_ij this is
// data dependent: ~8 (S + 2) 2^(-5S) for rows and columns without a wide
// spread of magnitudes (uniform data), much more where a row's largest entry
// dwarfs the entries that meet the column's mass.  The accuracy gate (on by
// default) bounds P_ij = (|A||B|)_ij 2^-(sigma_i + tau_j) from below with one
// more e4m3 slice per operand (the scaled magnitudes truncated onto the e4m3
// grid) and one more tensor-core product per K chunk, and where any entry's
// bound could exceed 1e-14 sqrt(m) (|A||B|)_ij, recomputes C with the FP64
// FMA kernel.
//
// Data layout in the library's scratch ("pack region" first, 128-byte rows,
// as the tensor-core kernel's tensor map requires):
//   A digits of chunk c: tile (mt, slice t, kb) at rows
//       a0_c + ((mt*SS + t)*kt_c + kb)*128, one row per row of A (128 k);
//   B digits of chunk c: tile (nt, slot, kb) at rows
//       b0_c + ((nt*SS + slot)*kt_c + kb)*bn, slot = S-1-u for slice u, one
//       row per column of B, so that B's slices L..0 are contiguous;
//   SS = S, or S + 1 with the gate, whose slice is t = slot = S;
//   then the row/column maxima (bit patterns), zero scale words, the level
//   sums D (FP32, [chunk][level] planes of n x p, padded so that planes are
//   not a power of two apart) followed by the gate's planes [chunk], the
//   problem table with the work units of each CTA, the unit map and the
//   gate's flag.
// The level problem (c, L) reads A's K blocks [0, (L+1) kt_c) and B's
// [(S-1-L) kt_c, S kt_c) of each tile through the table's K stride SS kt_c;
// the gate's problem c reads [S kt_c, (S+1) kt_c) of both.
// Rows (columns) holding a NaN or an infinity give NaN rows (columns) of C.
#include <cuda_fp8.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "ctx.h"
#include "split_common.cuh"

namespace mm {

constexpr int kOzakiMaxChunks = 1024;  // K chunks (the sum's int64 parts stay exact)

namespace {

constexpr int kRowsPerItem = 8;   // maxima: warps per block, one row of A each
constexpr int kColStrip = 32;     // maxima: columns of B per strip
constexpr int kRowChunk = 256;    // maxima: rows of B per strip item
constexpr int kSeg = 16;          // digits: consecutive k per thread

__device__ __forceinline__ uint64_t abs_bits64(double x) {
  return (uint64_t)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

// sigma = ilogb(max) + 2 from the bit pattern of a row's largest magnitude;
// 0 for an all-zero row; finite = false for a NaN or an infinity.
__device__ __forceinline__ int slice_exponent(uint64_t max_bits, bool &finite) {
  const int e_raw = (int)(max_bits >> 52);
  finite = e_raw != 0x7ff;
  if (max_bits == 0 || !finite) return 0;
  if (e_raw == 0) return (63 - __clzll((long long)max_bits)) - 1074 + 2;  // subnormal
  return e_raw - 1023 + 2;
}

// Truncated fixed-point magnitude F = floor(|x| 2^(5S - sigma)) (< 2^(5S-1)
// for |x| < 2^(sigma-1)) and the sign of x.
__device__ __forceinline__ uint64_t fixed_magnitude(double x, int sigma, int S, bool &neg) {
  const uint64_t bits = (uint64_t)__double_as_longlong(x);
  neg = (bits >> 63) != 0;
  const int e_raw = (int)((bits >> 52) & 0x7ff);
  const uint64_t frac = bits & 0xfffffffffffffull;
  uint64_t mant;
  int ex;
  if (e_raw == 0) {
    mant = frac;
    ex = -1022;
  } else {
    mant = frac | (1ull << 52);
    ex = e_raw - 1023;
  }
  const int sh = ex - 52 + 5 * S - sigma;  // |x| = mant 2^(ex - 52)
  if (mant == 0 || sh <= -64) return 0;
  return sh >= 0 ? (mant << sh) : (mant >> -sh);
}

// G = F + 16 (32^S - 1) / 31: 16 added to every base-32 position of F, so
// that g_t - 16 are the balanced digits (below 2^60 for S <= 12).
template <int S>
__device__ __forceinline__ uint64_t balanced_offset() {
  static_assert(S >= 2 && S <= 12, "slices");
  uint64_t o = 0;
#pragma unroll
  for (int t = 0; t < S; t++) o = (o << 5) | 16u;
  return o;
}

// 16 digits of slice t (one per k) from G -> 16 e4m3 bytes: d = g_t - 16
// (g_t = (G >> shift) & 31, the top slice unmasked), with the sign of x;
// zero digits are +0.
__device__ __forceinline__ uint4 digit_bytes(const uint64_t (&G)[kSeg], uint32_t negmask, int shift,
                                             bool top) {
  uint32_t w[4];
#pragma unroll
  for (int q = 0; q < 4; q++) {
    float v[4];
#pragma unroll
    for (int e = 0; e < 4; e++) {
      const uint64_t g = G[4 * q + e] >> shift;
      const int d = (int)(top ? g : (g & 31u)) - 16;
      v[e] = ((negmask >> (4 * q + e)) & 1u) && d ? -(float)d : (float)d;
    }
    const __nv_fp8x2_storage_t lo = __nv_cvt_float2_to_fp8x2(make_float2(v[0], v[1]), __NV_SATFINITE, __NV_E4M3);
    const __nv_fp8x2_storage_t hi = __nv_cvt_float2_to_fp8x2(make_float2(v[2], v[3]), __NV_SATFINITE, __NV_E4M3);
    w[q] = (uint32_t)lo | ((uint32_t)hi << 16);
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

// The accuracy gate's slice: 16 |x| 2^-sigma truncated toward zero onto the
// e4m3 grid (4 significant bits at 2^-6 and above, multiples of 2^-9 below;
// 0 under 2^-9), so the value is exact in e4m3 and never above 16 |x| 2^-sigma.
// Formed from the truncated fixed-point magnitude F = floor(|x| 2^(5S-sigma))
// in integer and FP32 arithmetic (16 |x| 2^-sigma >= F 2^(4-5S)): F's top four
// bits times a power of two (below 8, since |x| 2^-sigma < 1/2).
__device__ __forceinline__ float gate_value(uint64_t F, int S) {
  if (F == 0) return 0.0f;
  const int b = 64 - __clzll((long long)F);  // bit length, 1..5S-1
  const int sh = b > 4 ? b - 4 : 0;
  const float top = (float)(uint32_t)(F >> sh);  // 1..15, exact
  // 2^(sh + 4 - 5S) >= 2^(4 - 60): a normal float
  const float v = top * __int_as_float((sh + 4 - 5 * S + 127) << 23);
  return v >= 0x1p-6f ? v : floorf(v * 512.0f) * 0x1p-9f;
}

// 16 gate values -> 16 e4m3 bytes (exact conversions).
__device__ __forceinline__ uint4 gate_bytes(const float (&g)[kSeg]) {
  uint32_t w[4];
#pragma unroll
  for (int q = 0; q < 4; q++) {
    const __nv_fp8x2_storage_t lo =
        __nv_cvt_float2_to_fp8x2(make_float2(g[4 * q], g[4 * q + 1]), __NV_SATFINITE, __NV_E4M3);
    const __nv_fp8x2_storage_t hi =
        __nv_cvt_float2_to_fp8x2(make_float2(g[4 * q + 2], g[4 * q + 3]), __NV_SATFINITE, __NV_E4M3);
    w[q] = (uint32_t)lo | ((uint32_t)hi << 16);
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

// Maxima: items [0, ceil(n/8)) take 8 rows of A (a warp per row); the rest
// strips of 32 columns x 256 rows of B, merged into colmax with atomicMax on
// the bit patterns (which order like the magnitudes).
__global__ void __launch_bounds__(256)
ozaki_max_kernel(const double *__restrict__ A, const double *__restrict__ B, int64_t n, int64_t m,
                 int64_t p, uint64_t *__restrict__ rowmax, unsigned long long *__restrict__ colmax) {
  const int64_t items_a = (n + kRowsPerItem - 1) / kRowsPerItem;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if ((int64_t)blockIdx.x < items_a) {
    const int64_t i = (int64_t)blockIdx.x * kRowsPerItem + warp;
    if (i >= n) return;
    const double *row = A + i * m;
    uint64_t mx = 0;
    for (int64_t k = lane; k < m; k += 32) {
      const uint64_t b = abs_bits64(row[k]);
      mx = b > mx ? b : mx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const uint64_t other = __shfl_xor_sync(0xffffffffu, mx, o);
      mx = other > mx ? other : mx;
    }
    if (lane == 0) rowmax[i] = mx;
    return;
  }
  __shared__ uint64_t part[8][kColStrip];
  const int64_t b = (int64_t)blockIdx.x - items_a;
  const int64_t strips = (p + kColStrip - 1) / kColStrip;
  const int64_t c0 = (b % strips) * kColStrip, r0 = (b / strips) * kRowChunk;
  const int64_t col = c0 + lane;
  uint64_t mx = 0;
  if (col < p)
    for (int r = warp; r < kRowChunk; r += 8) {
      const int64_t k = r0 + r;
      if (k < m) {
        const uint64_t v = abs_bits64(B[k * p + col]);
        mx = v > mx ? v : mx;
      }
    }
  part[warp][lane] = mx;
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int w = 1; w < 8; w++) mx = part[w][lane] > mx ? part[w][lane] : mx;
    if (col < p) atomicMax(&colmax[col], (unsigned long long)mx);
  }
}

// A digits of one K chunk [k0, k0 + mc): one block per tile (mt, kb); a
// thread takes 16 consecutive k of a row (8 threads per 128-k row, 4 rows per
// warp: a warp's 16 loads read four whole 1 KB row segments, and each digit
// store instruction writes four whole 128-byte pack rows).  SS = S slices per
// tile, or S + 1 with the accuracy gate's slice (gate_value) after them.
template <int S>
__global__ void __launch_bounds__(256)
ozaki_digits_a_kernel(const double *__restrict__ A, int64_t n, int64_t m, int64_t k0, int64_t mc,
                      int kt, int SS, const uint64_t *__restrict__ rowmax,
                      uint4 *__restrict__ pack, int64_t a0) {
  const int mt = blockIdx.x / kt, kb = blockIdx.x % kt;
#pragma unroll 1
  for (int q = threadIdx.x; q < kTcBM * (128 / kSeg); q += 256) {
    const int r = q / (128 / kSeg), sg = q % (128 / kSeg);
    const int64_t i = (int64_t)mt * kTcBM + r;
    uint64_t F[kSeg];
    float Gv[kSeg];
    uint32_t negmask = 0;
    bool finite = true;
    const int sigma = i < n ? slice_exponent(rowmax[i], finite) : 0;
#pragma unroll
    for (int e = 0; e < kSeg; e++) {
      const int64_t kk = (int64_t)kb * 128 + sg * kSeg + e;  // within the chunk
      F[e] = 0;
      Gv[e] = 0.0f;
      if (i < n && finite && kk < mc) {
        bool neg;
        F[e] = fixed_magnitude(A[i * m + k0 + kk], sigma, S, neg);
        negmask |= (uint32_t)neg << e;
        if (SS > S) Gv[e] = gate_value(F[e], S);
      }
      F[e] += balanced_offset<S>();  // padding and zeros: all digits 0
    }
#pragma unroll
    for (int t = 0; t < S; t++) {
      const int64_t row = a0 + (((int64_t)mt * SS + t) * kt + kb) * kTcBM + r;
      pack[row * (kPackRowBytes / 16) + sg] = digit_bytes(F, negmask, 5 * (S - 1 - t), t == 0);
    }
    if (SS > S) {
      const int64_t row = a0 + (((int64_t)mt * SS + S) * kt + kb) * kTcBM + r;
      pack[row * (kPackRowBytes / 16) + sg] = gate_bytes(Gv);
    }
  }
}

// B digits of one K chunk: one block per tile (nt, kb); the bn columns are
// transposed through shared memory 32 at a time (FP64 rows of 32 columns
// read whole), then a thread takes 16 consecutive k of a column.
template <int S>
__global__ void __launch_bounds__(256)
ozaki_digits_b_kernel(const double *__restrict__ B, int64_t m, int64_t p, int64_t k0, int64_t mc,
                      int kt, int SS, int bn, const unsigned long long *__restrict__ colmax,
                      uint4 *__restrict__ pack, int64_t b0) {
  __shared__ double tile[128][32 + 1];
  const int nt = blockIdx.x / kt, kb = blockIdx.x % kt;
  const int tid = threadIdx.x;
  for (int c0 = 0; c0 < bn; c0 += 32) {
    for (int q = tid; q < 128 * 32; q += 256) {
      const int kk = q / 32, c = q % 32;
      const int64_t k = (int64_t)kb * 128 + kk, j = (int64_t)nt * bn + c0 + c;
      tile[kk][c] = (k < mc && j < p) ? B[(k0 + k) * p + j] : 0.0;
    }
    __syncthreads();
    {
      const int c = tid % 32, sg = tid / 32;  // 32 columns x 8 segments of 16 k
      const int64_t j = (int64_t)nt * bn + c0 + c;
      bool finite = true;
      const int tau = j < p ? slice_exponent(colmax[j], finite) : 0;
      uint64_t F[kSeg];
      float Gv[kSeg];
      uint32_t negmask = 0;
#pragma unroll
      for (int e = 0; e < kSeg; e++) {
        F[e] = 0;
        Gv[e] = 0.0f;
        if (j < p && finite) {
          bool neg;
          F[e] = fixed_magnitude(tile[sg * kSeg + e][c], tau, S, neg);
          negmask |= (uint32_t)neg << e;
          if (SS > S) Gv[e] = gate_value(F[e], S);
        }
        F[e] += balanced_offset<S>();  // padding and zeros: all digits 0
      }
#pragma unroll
      for (int u = 0; u < S; u++) {
        const int64_t row = b0 + (((int64_t)nt * SS + (S - 1 - u)) * kt + kb) * bn + c0 + c;
        pack[row * (kPackRowBytes / 16) + sg] = digit_bytes(F, negmask, 5 * (S - 1 - u), u == 0);
      }
      if (SS > S) {
        const int64_t row = b0 + (((int64_t)nt * SS + S) * kt + kb) * bn + c0 + c;
        pack[row * (kPackRowBytes / 16) + sg] = gate_bytes(Gv);
      }
    }
    __syncthreads();
  }
}

// The double nearest to hi:lo (ties to even), times 2^k.
__device__ __forceinline__ double int128_scaled(uint64_t lo, int64_t hi, int k) {
  const bool neg = hi < 0;
  uint64_t mlo = lo, mhi = (uint64_t)hi;
  if (neg) {  // magnitude
    mlo = ~lo + 1;
    mhi = ~(uint64_t)hi + (mlo == 0 ? 1 : 0);
  }
  double d;
  if (mhi == 0) {
    d = __ull2double_rn(mlo);
  } else {
    // keep the top 64 bits, with the bits shifted out as a sticky bit far
    // below the 53-bit rounding position, then round once
    const int sh = 64 - __clzll((long long)mhi);  // 1..64
    const uint64_t top = sh == 64 ? mhi : ((mhi << (64 - sh)) | (mlo >> sh));
    const uint64_t lost = sh == 64 ? mlo : (mlo << (64 - sh));
    d = __ull2double_rn(top | (lost != 0 ? 1ull : 0ull));
    k += sh;
  }
  d = neg ? -d : d;
  // times 2^k: one multiplication by the power of two when it is a normal
  // double (correctly rounded, as scalbn), scalbn otherwise
  if (k >= -1022 && k <= 1023) return d * __longlong_as_double((long long)(k + 1023) << 52);
  return scalbn(d, k);
}

// Item map of the level problems: unit u belongs to problem u / T (T tiles
// each, contiguous).
__global__ void __launch_bounds__(256)
ozaki_map_kernel(int *__restrict__ map, int64_t units, int64_t tiles) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u < units) map[u] = (int)(u / tiles);
}

// Both digit kernels of one K chunk, instantiated per S (the slice loops
// unroll with constant shifts).
cudaError_t launch_ozaki_digits(int S, int64_t blocks_a, int64_t blocks_b, cudaStream_t s,
                                const double *A, const double *B, int64_t n, int64_t m,
                                int64_t p, int64_t k0, int64_t mc, int kt, int SS, int bn,
                                const uint64_t *rowmax, const unsigned long long *colmax,
                                uint4 *pack, int64_t a0, int64_t b0) {
  if (blocks_a > 0x7fffffffLL || blocks_b > 0x7fffffffLL) return cudaErrorInvalidValue;
  switch (S) {
#define MM_OZ_DIG(V)                                                                            \
  case V:                                                                                       \
    ozaki_digits_a_kernel<V><<<(unsigned)blocks_a, 256, 0, s>>>(A, n, m, k0, mc, kt, SS, rowmax, \
                                                                pack, a0);                      \
    ozaki_digits_b_kernel<V><<<(unsigned)blocks_b, 256, 0, s>>>(B, m, p, k0, mc, kt, SS, bn,    \
                                                                colmax, pack, b0);              \
    break;
    MM_OZ_DIG(2) MM_OZ_DIG(3) MM_OZ_DIG(4) MM_OZ_DIG(5) MM_OZ_DIG(6) MM_OZ_DIG(7) MM_OZ_DIG(8)
    MM_OZ_DIG(9) MM_OZ_DIG(10) MM_OZ_DIG(11) MM_OZ_DIG(12)
#undef MM_OZ_DIG
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// The double nearest to M 2^k (M > 0 a 128-bit integer; ties to even) in
// integer arithmetic: the top 53 bits of M, rounded on the bits below them,
// and the exponent placed directly.  Returns false where the result is not a
// normal double (the caller then takes int128_scaled).
__device__ __forceinline__ bool round_to_double(unsigned __int128 M, int k, uint64_t &bits) {
  const uint64_t mh = (uint64_t)(M >> 64), ml = (uint64_t)M;
  const int L = mh ? 128 - __clzll((long long)mh) : 64 - __clzll((long long)ml);  // bit length
  int e = L - 1 + k;
  uint64_t top;
  if (L <= 53) {
    top = ml << (53 - L);  // exact
  } else {
    const int sh = L - 53;  // 1..75
    top = (uint64_t)(M >> sh);
    const unsigned __int128 rem = M - ((unsigned __int128)top << sh);
    const unsigned __int128 half = (unsigned __int128)1 << (sh - 1);
    if (rem > half || (rem == half && (top & 1u))) {
      if (++top == (1ull << 53)) {
        top >>= 1;
        e++;
      }
    }
  }
  if (e < -1022 || e > 1023) return false;
  bits = ((uint64_t)(e + 1023) << 52) | (top & ((1ull << 52) - 1));
  return true;
}

// c_ij = 2^(sigma_i + tau_j - 5(S+1)) sum_c sum_L D[c][L][i][j] 32^(S-1-L):
// the level sums are integers below 2^24, so their weighted sum is formed
// exactly in 128-bit integers and rounded once to FP64 (then scaled by a
// power of two, which rounds again only in the subnormal range); NaN where
// row i of A or column j of B is not finite.  A thread takes column j of the
// rows blockIdx.y, blockIdx.y + gridDim.y, ...; the S level values of a chunk
// are loaded together.  One instantiation per S, so the level loop unrolls
// without predicates.  The epilogue epi is applied to each entry; skip_if
// (the accuracy gate's flag, when given) set: the FP64 FMA product writes C
// instead and this kernel writes nothing.
template <int S>
__global__ void __launch_bounds__(256, 4)
ozaki_sum_kernel(const float *__restrict__ D, int64_t plane, int64_t n, int64_t p, int chunks,
                 const uint64_t *__restrict__ rowmax, const unsigned long long *__restrict__ colmax,
                 double *C, const int *skip_if, EpiT<double> epi) {
  if (skip_if != nullptr && *reinterpret_cast<const volatile int *>(skip_if) != 0) return;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= p) return;
  bool fb;
  const int tau = slice_exponent(colmax[j], fb);
  // Horner by 32 over levels 0..h-1 into X and h..S-1 into Y (int64: each
  // part at most (2^24 - 1)(32^6 - 1)/31 < 2^49.1 per chunk, below 2^63 over
  // at most kOzakiMaxChunks = 2^10 chunks), then v = X 32^(S-h) + Y once in
  // 128 bits
  constexpr int h = (S + 1) / 2;
  for (int64_t i = blockIdx.y; i < n; i += gridDim.y) {
    bool fa;
    const int sigma = slice_exponent(rowmax[i], fa);
    const int64_t x = i * p + j;
    int64_t X = 0, Y = 0;
    for (int c = 0; c < chunks; c++) {
      const float *d = D + (int64_t)c * S * plane + x;
      float v[S];
#pragma unroll
      for (int L = 0; L < S; L++) v[L] = __ldcs(d + (int64_t)L * plane);
      int64_t xc = 0, yc = 0;
#pragma unroll
      for (int L = 0; L < S; L++) {
        const int64_t q = __float2int_rn(v[L]);
        if (L < h) xc = xc * 32 + q;
        else yc = yc * 32 + q;
      }
      X += xc;
      Y += yc;
    }
    constexpr int sh = 5 * (S - h);  // 5..30
    uint64_t lo = (uint64_t)X << sh;
    int64_t hi = X >> (64 - sh);
    const uint64_t r = lo + (uint64_t)Y;
    hi += (Y < 0 ? -1 : 0) + (r < lo ? 1 : 0);
    lo = r;
    const int k = sigma + tau - 5 * (S + 1);
    double out;
    if (!(fa && fb)) {
      out = __longlong_as_double(0x7ff8000000000000ll);
    } else {
      const bool neg = hi < 0;
      unsigned __int128 M = ((unsigned __int128)(uint64_t)hi << 64) | lo;
      if (neg) M = ~M + 1;
      uint64_t bits;
      if (M == 0) out = 0.0;
      else if (round_to_double(M, k, bits)) out = __longlong_as_double((long long)(bits | ((uint64_t)neg << 63)));
      else out = int128_scaled(lo, hi, k);
    }
    C[x] = epi_apply(epi, out, x);
  }
}

cudaError_t launch_ozaki_sum(int S, dim3 grid, cudaStream_t s, const float *D, int64_t plane,
                             int64_t n, int64_t p, int chunks, const uint64_t *rowmax,
                             const unsigned long long *colmax, double *C, const int *skip_if,
                             const EpiT<double> &epi) {
  switch (S) {
#define MM_OZ_SUM(V) \
  case V: \
    ozaki_sum_kernel<V><<<grid, 256, 0, s>>>(D, plane, n, p, chunks, rowmax, colmax, C, skip_if, epi); \
    break;
    MM_OZ_SUM(2) MM_OZ_SUM(3) MM_OZ_SUM(4) MM_OZ_SUM(5) MM_OZ_SUM(6) MM_OZ_SUM(7) MM_OZ_SUM(8)
    MM_OZ_SUM(9) MM_OZ_SUM(10) MM_OZ_SUM(11) MM_OZ_SUM(12)
#undef MM_OZ_SUM
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Accuracy gate.  Every term a_ir b_rj of the emulated product is off by at
// most (S + 2) 2^(sigma_i + tau_j - 5S - 1), so entry (i, j) is off by at most
// m (S + 2) 2^(sigma_i + tau_j - 5S - 1); the product meets e_ij <= 1e-14 sqrt(m)
// wherever P_ij = sum_r |a_ir| 2^-sigma_i |b_rj| 2^-tau_j is at least
// sqrt(m) (S + 2) 2^(-5S-1) 1e14.  A lower bound of 256 P comes from the
// emulation's own machinery: one more slice per operand holds gate_value
// (16 |x| 2^-sigma truncated toward zero onto the e4m3 grid), and one more
// tensor-core product per K chunk multiplies the two (products exact in
// FP32; the FP32 accumulation of nonnegative terms is off by at most m 2^-23
// relative, which the host's threshold absorbs: it divides by 0.98 - m 2^-23,
// the 2% also covering the final rounding to a double, 2^-53 relative, below
// 1.2% of 1e-14; where m 2^-23 reaches 1/2 the threshold is infinite and
// every product falls back).  Truncation only lowers the bound, so entries
// whose magnitudes fall below the e4m3 grid cause a fallback, never a miss.
// The check kernel adds the chunks' planes in FP32 (at most 1024 nonnegative
// terms), lowers the sum by 2^-10 (more than that addition's rounding) and
// sets a flag where any entry with a finite, non-zero row and column misses
// the threshold; the FP64 FMA product then recomputes C.
__global__ void __launch_bounds__(256)
ozaki_gate_check_kernel(const float *__restrict__ G, int64_t plane, int chunks, int64_t n,
                        int64_t p, const uint64_t *__restrict__ rowmax,
                        const unsigned long long *__restrict__ colmax, float thr256, int *flag) {
  bool fail = false;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    bool fi;
    slice_exponent(rowmax[i], fi);
    // a row with a NaN or an infinity gives NaN by design; an all-zero row
    // gives exact zeros
    if (!fi || rowmax[i] == 0) continue;
    for (int64_t j = threadIdx.x; j < p; j += blockDim.x) {
      bool fj;
      slice_exponent(colmax[j], fj);
      if (!fj || colmax[j] == 0) continue;
      float v = 0.0f;
      for (int c = 0; c < chunks; c++) v += __ldcs(G + (int64_t)c * plane + i * p + j);
      if (!(v * (1.0f - 0x1p-10f) >= thr256)) fail = true;
    }
  }
  if (__syncthreads_or(fail) && threadIdx.x == 0) atomicOr(flag, 1);
}

// Scratch offsets of one call.
struct OzLayout {
  int S, SS, chunks, bn, mt, nt;
  int64_t mc;
  std::vector<int64_t> k0, kc, kt, a0, b0;
  int64_t rows = 0, plane = 0;
  size_t max_off, zero_off, zero_end, d_off, tab_off, map_off, flag_off, simt_off, need;
  int64_t units = 0;
};

}  // namespace

int64_t ozaki_chunk(int S) {
  const int64_t mc = ((int64_t)((1 << 24) - 1) / (256 * (int64_t)S)) / 128 * 128;
  return mc;
}

mm_status run_ozaki(Scratch &ws, int64_t n, int64_t m, int64_t p, const double *A,
                    const double *B, double *C, int S, bool gate, cudaStream_t s, const Epi *epi) {
  if (S < kOzakiMinSlices || S > kOzakiMaxSlices) return MM_EINVAL;
  if (n == 0 || p == 0) return MM_OK;
  if (m == 0) return note_cuda(cudaMemsetAsync(C, 0, (size_t)(n * p) * sizeof(double), s));
  OzLayout lay;
  lay.S = S;
  lay.SS = S + (gate ? 1 : 0);  // slices per tile in the packs (the gate's last)
  lay.mc = ozaki_chunk(S);
  if (ceil_div(m, lay.mc) > kOzakiMaxChunks) return MM_EINVAL;
  lay.chunks = (int)ceil_div(m, lay.mc);
  TcChoice ch = tune_choose(n, std::min(m, lay.mc), p);
  lay.bn = tc_bn(kTcE4m3, ch.bn);
  lay.mt = (int)ceil_div(n, kTcBM);
  lay.nt = (int)ceil_div(p, lay.bn);
  for (int c = 0; c < lay.chunks; c++) {
    const int64_t k0 = (int64_t)c * lay.mc, kc = std::min(lay.mc, m - k0);
    const int64_t kt = ceil_div(kc, 128);
    lay.k0.push_back(k0);
    lay.kc.push_back(kc);
    lay.kt.push_back(kt);
    lay.a0.push_back(lay.rows);
    lay.rows += (int64_t)lay.mt * lay.SS * kt * kTcBM;
    lay.b0.push_back(lay.rows);
    lay.rows += (int64_t)lay.nt * lay.SS * kt * lay.bn;
  }
  if (lay.rows > 0x7fffffffLL) return MM_EINVAL;
  // S level problems per chunk, then the gate's product per chunk
  const int nprobs = lay.chunks * lay.SS;
  const int64_t tiles = (int64_t)lay.mt * lay.nt;
  // level planes of D, padded so that the planes of one entry do not sit a
  // power of two apart (128-byte aligned)
  lay.plane = (n * p + 31) / 32 * 32 + 32;
  std::vector<SplitProb> tab((size_t)nprobs);
  // level problems, longest K first (the persistent grid takes units in
  // order, so the short ones fill the last wave); problem g = (S-1-L) *
  // chunks + c holds units [g T, (g+1) T) of the T tiles.  (Interleaving the
  // levels tile by tile was measured slower: 19 GB of DRAM reads per 4096^3
  // launch instead of 11, 5.4 ms instead of 4.6.)
  int g = 0;
  for (int L = S - 1; L >= 0; L--)
    for (int c = 0; c < lay.chunks; c++, g++) {
      SplitProb &sp = tab[(size_t)g];
      std::memset(&sp, 0, sizeof(sp));
      const int64_t kt = lay.kt[(size_t)c];
      sp.n = (int32_t)n;
      sp.p = (int32_t)p;
      sp.kt = (int32_t)((L + 1) * kt);
      sp.m = sp.kt * 128;  // padded K of the level: zero digits past the chunk
      sp.mt = lay.mt;
      sp.nt = lay.nt;
      sp.bn = lay.bn;
      sp.group_m = ch.group_m;
      sp.a_row0 = lay.a0[(size_t)c];
      sp.b_row0 = lay.b0[(size_t)c] + (int64_t)(S - 1 - L) * kt * lay.bn;
      sp.a_kstride = (int32_t)(lay.SS * kt);
      sp.b_kstride = (int32_t)(lay.SS * kt);
      sp.unit_start = (int32_t)lay.units;
      lay.units += tiles;
      sp.split_from = (int32_t)tiles;
      sp.split_s = 1;
      sp.C = reinterpret_cast<float *>((uintptr_t)(((int64_t)c * S + L) * lay.plane));  // offset
    }
  // the gate's products (one slice against one slice: as short as level 0,
  // so they run last), planes after the level planes
  for (int c = 0; gate && c < lay.chunks; c++, g++) {
    SplitProb &sp = tab[(size_t)g];
    std::memset(&sp, 0, sizeof(sp));
    const int64_t kt = lay.kt[(size_t)c];
    sp.n = (int32_t)n;
    sp.p = (int32_t)p;
    sp.kt = (int32_t)kt;
    sp.m = sp.kt * 128;
    sp.mt = lay.mt;
    sp.nt = lay.nt;
    sp.bn = lay.bn;
    sp.group_m = ch.group_m;
    sp.a_row0 = lay.a0[(size_t)c] + (int64_t)S * kt * kTcBM;
    sp.b_row0 = lay.b0[(size_t)c] + (int64_t)S * kt * lay.bn;
    sp.a_kstride = (int32_t)(lay.SS * kt);
    sp.b_kstride = (int32_t)(lay.SS * kt);
    sp.unit_start = (int32_t)lay.units;
    lay.units += tiles;
    sp.split_from = (int32_t)tiles;
    sp.split_s = 1;
    sp.C = reinterpret_cast<float *>((uintptr_t)(((int64_t)lay.chunks * S + c) * lay.plane));
  }
  if (lay.units > 0x7fffffffLL) return MM_EINVAL;
  const size_t pack_bytes = (size_t)lay.rows * kPackRowBytes;
  lay.max_off = (pack_bytes + 255) & ~(size_t)255;  // row maxima (n) + column maxima (p)
  lay.zero_off = lay.max_off;
  lay.zero_end = lay.max_off + (size_t)(n + p) * 8 + (size_t)(n + p) * 4;  // + zero scale words
  lay.d_off = (lay.zero_end + 255) & ~(size_t)255;
  lay.tab_off = (lay.d_off + (size_t)nprobs * lay.plane * sizeof(float) + 255) & ~(size_t)255;
  // the table, then the work units of each CTA (the levels differ in length)
  TcConfig cfg{128, 4, ch.grid};
  cfg.max_bn = lay.bn;
  std::vector<int> order;
  tc_unit_order(tab.data(), nprobs, tc_launch_grid(cfg, lay.units), order);
  const size_t tab_bytes = ((size_t)nprobs * sizeof(SplitProb) + 15) & ~(size_t)15;
  lay.map_off = (lay.tab_off + tab_bytes + order.size() * sizeof(int) + 255) & ~(size_t)255;
  // the gate's fallback flag
  lay.flag_off = (lay.map_off + (size_t)lay.units * sizeof(int) + 255) & ~(size_t)255;
  // the fallback's K-slice partials (under-filled products)
  lay.simt_off = lay.flag_off + 256;
  lay.need = lay.simt_off + simt_scratch_bytes(true, n, m, p);
  cudaError_t e = ws.reserve(lay.need, s);
  if (e != cudaSuccess) return note_cuda(e);
  uint8_t *base = static_cast<uint8_t *>(ws.ptr);
  uint64_t *rowmax = reinterpret_cast<uint64_t *>(base + lay.max_off);
  unsigned long long *colmax = reinterpret_cast<unsigned long long *>(rowmax + n);
  uint32_t *zero_words = reinterpret_cast<uint32_t *>(colmax + p);
  float *D = reinterpret_cast<float *>(base + lay.d_off);
  for (auto &sp : tab) {
    sp.C = D + (uintptr_t)sp.C;
    sp.sA = zero_words;      // scale exponent 0: the digits are not rescaled
    sp.tB = zero_words + n;
  }
  SplitProb *d_tab = reinterpret_cast<SplitProb *>(base + lay.tab_off);
  const int *d_order = reinterpret_cast<const int *>(base + lay.tab_off + tab_bytes);
  {
    std::vector<uint8_t> blob(tab_bytes + order.size() * sizeof(int), 0);
    std::memcpy(blob.data(), tab.data(), tab.size() * sizeof(SplitProb));
    std::memcpy(blob.data() + tab_bytes, order.data(), order.size() * sizeof(int));
    e = ws.stage.copy_to_device(d_tab, blob.data(), blob.size(), s);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(base + lay.zero_off, 0, lay.zero_end - lay.zero_off, s);
  if (e != cudaSuccess) return note_cuda(e);
  {
    TraceScope ts("ozaki_max", s);
    const int64_t items = ceil_div(n, kRowsPerItem) + ceil_div(p, kColStrip) * ceil_div(m, kRowChunk);
    if (items > 0x7fffffffLL) return MM_EINVAL;
    ozaki_max_kernel<<<(unsigned)items, 256, 0, s>>>(A, B, n, m, p, rowmax, colmax);
    if ((e = cudaGetLastError()) != cudaSuccess) return note_cuda(e);
  }
  {
    TraceScope ts("ozaki_digits", s);
    uint4 *pk = static_cast<uint4 *>(ws.ptr);
    for (int c = 0; c < lay.chunks; c++) {
      const int kt = (int)lay.kt[(size_t)c];
      e = launch_ozaki_digits(S, lay.mt * kt, lay.nt * kt, s, A, B, n, m, p, lay.k0[(size_t)c],
                              lay.kc[(size_t)c], kt, lay.SS, lay.bn, rowmax, colmax, pk,
                              lay.a0[(size_t)c], lay.b0[(size_t)c]);
      if (e != cudaSuccess) return note_cuda(e);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return note_cuda(e);
  }
  int *unit_map = reinterpret_cast<int *>(base + lay.map_off);
  {
    TraceScope ts("ozaki_map", s);
    ozaki_map_kernel<<<(unsigned)ceil_div(lay.units, 256), 256, 0, s>>>(unit_map, lay.units,
                                                                          tiles);
    if ((e = cudaGetLastError()) != cudaSuccess) return note_cuda(e);
  }
  e = launch_tc(kTcE4m3, d_tab, nprobs, (int)lay.units, unit_map, nullptr, ws.ptr, lay.rows, cfg,
                g_ctx.d_err, s, d_order);
  if (e != cudaSuccess) return note_cuda(e);
  // the gate reads the level sums only, so it runs before the sum kernel:
  // where it fails, the sum writes nothing and the FP64 FMA product below
  // reads the epilogue's D (which may be C) untouched
  int *flag = gate ? reinterpret_cast<int *>(base + lay.flag_off) : nullptr;
  if (gate) {
    TraceScope ts("ozaki_gate", s);
    if ((e = cudaMemsetAsync(flag, 0, sizeof(int), s)) != cudaSuccess) return note_cuda(e);
    const double room = 0.98 - (double)m * 0x1p-23;
    const double thr256 = room < 0.5 ? (double)INFINITY
                                     : 256.0 * std::sqrt((double)m) * (S + 2) *
                                           std::ldexp(1.0, -5 * S - 1) * 1e14 / room;
    float thr = (float)thr256;  // rounded up to a float
    if ((double)thr < thr256) thr = std::nextafter(thr, (float)INFINITY);
    const unsigned gc = (unsigned)std::min<int64_t>(n, (int64_t)sm_count() * 8);
    ozaki_gate_check_kernel<<<gc, 256, 0, s>>>(D + (int64_t)lay.chunks * S * lay.plane, lay.plane,
                                                lay.chunks, n, p, rowmax, colmax, thr, flag);
    if ((e = cudaGetLastError()) != cudaSuccess) return note_cuda(e);
  }
  {
    TraceScope ts("ozaki_sum", s);
    const int64_t gx = ceil_div(p, 256);
    // one wave: four blocks per SM (the launch bound)
    const int64_t gy = std::max<int64_t>(1, std::min<int64_t>({n, 65535, ceil_div((int64_t)sm_count() * 4, gx)}));
    if (gx > 0x7fffffffLL) return MM_EINVAL;
    e = launch_ozaki_sum(S, dim3((unsigned)gx, (unsigned)gy), s, D, lay.plane, n, p, lay.chunks,
                         rowmax, colmax, C, flag, epi_of<double>(epi));
    if (e != cudaSuccess) return note_cuda(e);
    if ((e = cudaGetLastError()) != cudaSuccess) return note_cuda(e);
  }
  if (!gate) return MM_OK;
  // the FP64 FMA product replaces C where the flag is set: the same kernels
  // and K slices as MM_MODE_DGEMM, so the bits are that mode's
  const SimtPlan pl = simt_plan(true, n, m, p);
  if (pl.S >= 1)
    return note_cuda(launch_simt_splitk_f64(
        n, m, p, A, B, C, pl.S > 1 ? reinterpret_cast<double *>(base + lay.simt_off) : nullptr, pl, s,
        flag, epi));
  return note_cuda(launch_simt_f64(n, m, p, A, B, C, s, flag, epi));
}

size_t ozaki_scratch_bytes(int64_t n, int64_t m, int64_t p, int S) {
  if (n <= 0 || p <= 0 || m <= 0) return 0;
  const int64_t mc = ozaki_chunk(S);
  const int64_t chunks = ceil_div(m, mc);
  const int64_t kt_all = ceil_div(m, 128) + chunks;  // K blocks over all chunks (bound)
  // S digit slices per operand and the accuracy gate's slice (counted whether
  // or not the gate is on), their level sums and the gate's planes, maxima,
  // table, the CTAs' unit lists and the unit map
  const int64_t SS = S + 1;
  const int64_t rows = (ceil_div(n, kTcBM) * kTcBM + ceil_div(p, 128) * 256) * SS * kt_all;
  return (size_t)rows * kPackRowBytes + (size_t)chunks * SS * (n * p + 64) * sizeof(float) +
         (size_t)(n + p) * 12 + (size_t)chunks * SS * ceil_div(n, kTcBM) * ceil_div(p, 128) * 4 +
         (size_t)chunks * SS * sizeof(SplitProb) +
         (size_t)chunks * SS * ceil_div(n, kTcBM) * ceil_div(p, 128) * 4 + ((size_t)1 << 20) +
         simt_scratch_bytes(true, n, m, p);
}

}  // namespace mm

extern "C" mm_status mm_ozaki_plan(int64_t n, int64_t m, int64_t p, int slices,
                                   int64_t *chunk_columns, int *chunks, size_t *scratch_bytes) {
  using namespace mm;
  if (n < 0 || m < 0 || p < 0 || slices < kOzakiMinSlices || slices > kOzakiMaxSlices ||
      !chunk_columns || !chunks || !scratch_bytes)
    return MM_EINVAL;
  const int64_t mc = ozaki_chunk(slices);
  const int64_t q = ceil_div(m, mc);
  if (q > kOzakiMaxChunks) return MM_EINVAL;
  *chunk_columns = mc;
  *chunks = (int)q;
  *scratch_bytes = ozaki_scratch_bytes(n, m, p, slices);
  return MM_OK;
}

namespace mm {

}  // namespace mm
