// Device helpers shared by the split-BF16x3 prep and tensor-core kernels.
#pragma once

#include <cuda_bf16.h>

#include "mm_internal.h"

namespace mm {

// x * 2^e rounded once: a multiplication by the exact power of two when 2^e is
// a normal float (then identical to ldexpf, which is exact to 0 ulp), ldexpf
// otherwise.
__device__ __forceinline__ float scale_pow2(float x, int e) {
  if (e >= -126 && e <= 127) return x * __int_as_float((e + 127) << 23);
  return ldexpf(x, e);
}

// Scale exponent of a row of A / column of B from the bit pattern of its
// largest magnitude: s = floor(log2(max |x|)), so that x * 2^-s has magnitude
// below 2 for every entry of the row/column.  An all-zero row and a
// non-finite maximum give s = 0 (non-finite values then propagate through
// the products as IEEE arithmetic would).
__device__ __forceinline__ int scale_exponent(uint32_t max_bits) {
  const float f = __uint_as_float(max_bits);
  if (!(f > 0.0f) || f > 3.402823466e38f) return 0;
  return ilogbf(f);
}

// Finds the problem whose [start, next start) range holds `item`: one load
// from the item -> problem map when there is one (tables of many problems),
// else a binary search over the start prefixes.
template <typename F>
__device__ __forceinline__ int find_problem(const SplitProb *__restrict__ probs, int nprobs,
                                            const int *__restrict__ map, int item, F start_of) {
  if (map) return map[item];
  int lo = 0, hi = nprobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (start_of(probs[mid]) <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

}  // namespace mm
