// FP64 check of a computed product on the GPU: the error-norm reduction that
// accompanies every result when checking is on.
//
// Freivalds' test (R. Freivalds, "Probabilistic machines can use less running
// time", IFIP 1977): for a random vector x, a correct C satisfies
// C.x = A.(B.x).  The kernels compute w = B.x, z = A.w, y = C.x in FP64 and
// the normalised residual max_i |y_i - z_i| / (|A|.(|B|.|x|))_i.
// Sampled entries: max_t |C_IJ - sum_r A_Ir B_rJ| / sum_r |A_Ir||B_rJ| for
// given positions (I_t, J_t), dot products in FP64.
#include "mm_internal.h"

namespace mm {
namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Non-negative doubles order like their bit patterns; NaN is mapped to +inf.
__device__ __forceinline__ void atomic_max_nonneg(double *dst, double v) {
  if (!(v == v)) v = __longlong_as_double(0x7ff0000000000000LL);
  atomicMax(reinterpret_cast<unsigned long long *>(dst),
            static_cast<unsigned long long>(__double_as_longlong(v)));
}

__device__ __forceinline__ double ratio(double diff, double norm) {
  if (norm > 0.0) return diff / norm;
  return diff == 0.0 ? 0.0 : __longlong_as_double(0x7ff0000000000000LL);
}

// w = B.x and wa = |B|.|x| (B: rows x cols), one warp per row.
template <typename T>
__global__ void __launch_bounds__(256)
check_gemv_kernel(const T *__restrict__ B, const double *__restrict__ x, int64_t rows,
                  int64_t cols, double *__restrict__ w, double *__restrict__ wa) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < rows; r += nwarps) {
    double s = 0.0, sa = 0.0;
    for (int64_t c = lane; c < cols; c += 32) {
      const double b = (double)B[r * cols + c];
      s = fma(b, x[c], s);
      sa = fma(fabs(b), fabs(x[c]), sa);
    }
    s = warp_sum(s);
    sa = warp_sum(sa);
    if (lane == 0) { w[r] = s; wa[r] = sa; }
  }
}

// Per row i of A and C: z = A_i.w, za = |A_i|.wa, y = C_i.x; out[0] = max ratio.
template <typename T>
__global__ void __launch_bounds__(256)
check_freivalds_kernel(const T *__restrict__ A, const T *__restrict__ C,
                       const double *__restrict__ x, const double *__restrict__ w,
                       const double *__restrict__ wa, int64_t n, int64_t m, int64_t p,
                       double *__restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double worst = 0.0;
  for (int64_t i = warp; i < n; i += nwarps) {
    double z = 0.0, za = 0.0, y = 0.0;
    for (int64_t k = lane; k < m; k += 32) {
      const double a = (double)A[i * m + k];
      z = fma(a, w[k], z);
      za = fma(fabs(a), wa[k], za);
    }
    for (int64_t j = lane; j < p; j += 32) y = fma((double)C[i * p + j], x[j], y);
    z = warp_sum(z);
    za = warp_sum(za);
    y = warp_sum(y);
    const double r = ratio(fabs(y - z), za);
    worst = (r > worst || !(r == r)) ? r : worst;
  }
  if (lane == 0) atomic_max_nonneg(out, worst);
}

// One warp per sampled entry: out[1] = max |C_IJ - (A.B)_IJ| / (|A|.|B|)_IJ.
template <typename T>
__global__ void __launch_bounds__(256)
check_samples_kernel(const T *__restrict__ A, const T *__restrict__ B, const T *__restrict__ C,
                     int64_t n, int64_t m, int64_t p, const int64_t *__restrict__ I,
                     const int64_t *__restrict__ J, int64_t count, double *__restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double worst = 0.0;
  for (int64_t t = warp; t < count; t += nwarps) {
    const int64_t i = I[t], j = J[t];
    if (i < 0 || i >= n || j < 0 || j >= p) { worst = __longlong_as_double(0x7ff0000000000000LL); continue; }
    double s = 0.0, sa = 0.0;
    for (int64_t k = lane; k < m; k += 32) {
      const double a = (double)A[i * m + k], b = (double)B[k * p + j];
      s = fma(a, b, s);
      sa = fma(fabs(a), fabs(b), sa);
    }
    s = warp_sum(s);
    sa = warp_sum(sa);
    const double r = ratio(fabs((double)C[i * p + j] - s), sa);
    worst = (r > worst || !(r == r)) ? r : worst;
  }
  if (lane == 0) atomic_max_nonneg(out + 1, worst);
}

template <typename T>
cudaError_t launch_check_t(int64_t n, int64_t m, int64_t p, const T *A, const T *B, const T *C,
                           const double *x, int64_t ns, const int64_t *I, const int64_t *J,
                           double *work, double *out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, 2 * sizeof(double), s);
  if (e != cudaSuccess) return e;
  const int blocks = sm_count() * 8;
  TraceScope ts("check_f64", s);
  if (m > 0) {
    check_gemv_kernel<T><<<blocks, 256, 0, s>>>(B, x, m, p, work, work + m);
  }
  check_freivalds_kernel<T><<<blocks, 256, 0, s>>>(A, C, x, work, work + m, n, m, p, out);
  if (ns > 0) check_samples_kernel<T><<<blocks, 256, 0, s>>>(A, B, C, n, m, p, I, J, ns, out);
  return cudaGetLastError();
}

}  // namespace

size_t check_work_doubles(int64_t n, int64_t m, int64_t p) {
  (void)n; (void)p;
  return (size_t)(2 * (m > 0 ? m : 1));
}

cudaError_t launch_check(bool f64, int64_t n, int64_t m, int64_t p, const void *A, const void *B,
                         const void *C, const double *x, int64_t nsamples, const int64_t *I,
                         const int64_t *J, double *d_work, double *d_out, cudaStream_t s) {
  if (f64)
    return launch_check_t<double>(n, m, p, (const double *)A, (const double *)B,
                                  (const double *)C, x, nsamples, I, J, d_work, d_out, s);
  return launch_check_t<float>(n, m, p, (const float *)A, (const float *)B, (const float *)C, x,
                               nsamples, I, J, d_work, d_out, s);
}

}  // namespace mm
