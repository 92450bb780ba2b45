// The paper's other workloads around the product, as bandwidth-bound kernels
// and a complex product built on the real paths.
//
//   mm_cgemm  complex C = A.B (Table 2's "complex float" column): the complex
//             operands are split into real and imaginary planes, the four real
//             products Ar.Br, Ai.Bi, Ar.Bi, Ai.Br run as one grouped call of
//             the chosen real path, and C = (Ar.Br - Ai.Bi) + i (Ar.Bi + Ai.Br)
//             is assembled.  Four products rather than three (Gauss) keep the
//             imaginary part free of the cancellation Gauss's form adds.
//   mm_add    C = alpha A + beta B elementwise: the matrix addition /
//             subtraction the paper also measures (results section).
//   mm_diag   C = X.diag(d) or diag(d).X: the diagonal special case the paper
//             names in the algorithms section, as a column/row scaling that
//             reads X once (O(n p) work instead of the dense O(n p k)).
#include <algorithm>

#include "ctx.h"

namespace mm {
namespace {

__global__ void __launch_bounds__(256)
cplx_planes_kernel(const float2 *__restrict__ z, float *__restrict__ re, float *__restrict__ im,
                   int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = z[i];
    re[i] = v.x;
    im[i] = v.y;
  }
}

// C = (P0 - P1) + i (P2 + P3), interleaved
__global__ void __launch_bounds__(256)
cplx_combine_kernel(const float *__restrict__ p0, const float *__restrict__ p1,
                    const float *__restrict__ p2, const float *__restrict__ p3,
                    float2 *__restrict__ c, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    c[i] = make_float2(p0[i] - p1[i], p2[i] + p3[i]);
}

template <typename T>
__global__ void __launch_bounds__(256)
add_kernel(const T *__restrict__ a, const T *__restrict__ b, T *__restrict__ c, T alpha, T beta,
           int64_t count, bool unit) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    // alpha = 1, beta = +-1: one correctly rounded addition or subtraction
    c[i] = unit ? a[i] + beta * b[i] : fma(alpha, a[i], beta * b[i]);
  }
}

// c = beta d (c may be d)
template <typename T>
__global__ void __launch_bounds__(256)
scale_kernel(const T *d, T *c, T beta, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    c[i] = beta * d[i];
}

// The 16-byte kernels below give each block one contiguous run of
// 256 * kEwUnroll vectors (thread t takes vectors t, t + 256, ...): all loads
// of a thread are issued before its stores, and consecutive blocks sweep
// memory in order.  (Measured on GB300 against a persistent grid-stride form
// of the same loop: 5.9 vs 5.5 TB/s at 4096^2, 7.2 vs 6.8 TB/s at 16384^2.)
constexpr int kEwUnroll = 4;
constexpr int kEwThreads = 256;

// 16-byte variant for aligned float operands
__global__ void __launch_bounds__(kEwThreads)
add4_kernel(const float4 *__restrict__ a, const float4 *__restrict__ b, float4 *__restrict__ c,
            float alpha, float beta, int64_t count4, bool unit) {
  auto op = [&](const float4 &x, const float4 &y) {
    if (unit)
      return make_float4(x.x + beta * y.x, x.y + beta * y.y, x.z + beta * y.z, x.w + beta * y.w);
    return make_float4(fmaf(alpha, x.x, beta * y.x), fmaf(alpha, x.y, beta * y.y),
                       fmaf(alpha, x.z, beta * y.z), fmaf(alpha, x.w, beta * y.w));
  };
  const int64_t base = (int64_t)blockIdx.x * kEwThreads * kEwUnroll + threadIdx.x;
  float4 x[kEwUnroll], y[kEwUnroll];
#pragma unroll
  for (int u = 0; u < kEwUnroll; u++) {
    const int64_t i = base + (int64_t)u * kEwThreads;
    if (i < count4) {
      x[u] = a[i];
      y[u] = b[i];
    }
  }
#pragma unroll
  for (int u = 0; u < kEwUnroll; u++) {
    const int64_t i = base + (int64_t)u * kEwThreads;
    if (i < count4) c[i] = op(x[u], y[u]);
  }
}

// side 0: C[i][j] = X[i][j] * d[j];  side 1: C[i][j] = d[i] * X[i][j].
// Scalar form: blocks stride over rows (y) and column chunks (x).
template <typename T>
__global__ void __launch_bounds__(256)
diag_kernel(const T *__restrict__ x, const T *__restrict__ d, T *__restrict__ c, int64_t n,
            int64_t p, int side) {
  for (int64_t r = blockIdx.y; r < n; r += gridDim.y) {
    const T dr = side == 1 ? d[r] : T(0);
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p;
         j += (int64_t)gridDim.x * blockDim.x) {
      const int64_t i = r * p + j;
      c[i] = x[i] * (side == 0 ? d[j] : dr);
    }
  }
}

// 16-byte form for aligned float operands with p % 4 == 0: vectors of the
// flat n * p4 range (p4 = p / 4) in the same contiguous runs as add4_kernel;
// each thread finds the (row, vector column) of its first vector and advances
// it by the block width's quotient and remainder, so no division runs per
// vector.
__global__ void __launch_bounds__(kEwThreads)
diag4_kernel(const float4 *__restrict__ x, const float *__restrict__ d, float4 *__restrict__ c,
             int64_t n, int64_t p4, int side) {
  const int64_t count4 = n * p4;
  const int64_t base = (int64_t)blockIdx.x * kEwThreads * kEwUnroll + threadIdx.x;
  const int64_t s_row = kEwThreads / p4, s_col = kEwThreads % p4;
  int64_t r = base / p4, j = base % p4;
  float4 v[kEwUnroll];
  int64_t rs[kEwUnroll], js[kEwUnroll];
#pragma unroll
  for (int u = 0; u < kEwUnroll; u++) {
    const int64_t i = base + (int64_t)u * kEwThreads;
    if (i < count4) v[u] = x[i];
    rs[u] = r;
    js[u] = j;
    r += s_row;
    j += s_col;
    if (j >= p4) {
      j -= p4;
      r++;
    }
  }
#pragma unroll
  for (int u = 0; u < kEwUnroll; u++) {
    const int64_t i = base + (int64_t)u * kEwThreads;
    if (i >= count4) continue;
    const float4 s4 = side == 0 ? __ldg(reinterpret_cast<const float4 *>(d) + js[u])
                                : make_float4(d[rs[u]], d[rs[u]], d[rs[u]], d[rs[u]]);
    c[i] = make_float4(v[u].x * s4.x, v[u].y * s4.y, v[u].z * s4.z, v[u].w * s4.w);
  }
}

// Grid of the 16-byte kernels: one block per run of 256 * kEwUnroll vectors.
int64_t grid_ew(int64_t count4) {
  const int64_t g = (count4 + (int64_t)kEwThreads * kEwUnroll - 1) / ((int64_t)kEwThreads * kEwUnroll);
  return g > 0 ? g : 1;
}

int grid_for(int64_t count) {
  const int64_t want = (count + 255) / 256;
  const int64_t cap = (int64_t)sm_count() * 16;
  return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace
}  // namespace mm

using namespace mm;

extern "C" {

mm_status mm_cgemm(int64_t n, int64_t m, int64_t p, const void *A, const void *B, void *C,
                   mm_mode mode) {
  if (!g_ctx.inited) return MM_ENOTINIT;
  if (g_ctx.sticky) return MM_ECUDA;
  if (n < 0 || m < 0 || p < 0) return MM_EINVAL;
  if (mode == MM_MODE_AUTO) mode = MM_MODE_SPLIT_BF16X3;
  if (mode != MM_MODE_SIMT && mode != MM_MODE_SPLIT_BF16X3) return MM_EUNSUPPORTED;
  if (n == 0 || p == 0) return MM_OK;
  if (!C || (m > 0 && (!A || !B))) return MM_EINVAL;
  if (pointer_kind(C) != 1 || (m > 0 && (pointer_kind(A) != 1 || pointer_kind(B) != 1)))
    return MM_EINVAL;
  std::lock_guard<std::mutex> lk(g_api_mutex);
  cudaStream_t s = g_ctx.stream;
  if (m == 0) return note_cuda(cudaMemsetAsync(C, 0, (size_t)(n * p) * 8, s)) == MM_OK
                         ? check_device_flag(s) : MM_ECUDA;
  // scratch: Ar, Ai (n x m), Br, Bi (m x p), four real products (n x p)
  const size_t na = (size_t)(n * m), nb = (size_t)(m * p), nc = (size_t)(n * p);
  auto up = [](size_t x) { return (x + 63) & ~(size_t)63; };
  const size_t total = 2 * up(na) + 2 * up(nb) + 4 * up(nc);
  cudaError_t e = g_ctx.cplx_ws.reserve(total * sizeof(float), s);
  if (e != cudaSuccess) return note_cuda(e);
  float *ar = static_cast<float *>(g_ctx.cplx_ws.ptr), *ai = ar + up(na);
  float *br = ai + up(na), *bi = br + up(nb);
  float *pr[4];
  pr[0] = bi + up(nb);
  for (int q = 1; q < 4; q++) pr[q] = pr[q - 1] + up(nc);
  {
    TraceScope ts("cplx_planes", s);
    cplx_planes_kernel<<<grid_for((int64_t)na), 256, 0, s>>>(static_cast<const float2 *>(A), ar, ai,
                                                             (int64_t)na);
  }
  {
    TraceScope ts("cplx_planes", s);
    cplx_planes_kernel<<<grid_for((int64_t)nb), 256, 0, s>>>(static_cast<const float2 *>(B), br, bi,
                                                             (int64_t)nb);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return note_cuda(e);
  const mm_problem probs[4] = {{n, m, p, ar, br, pr[0]}, {n, m, p, ai, bi, pr[1]},
                               {n, m, p, ar, bi, pr[2]}, {n, m, p, ai, br, pr[3]}};
  mm_status st = enqueue_grouped(g_ctx.split_ws, g_ctx.grouped_ws, 4, probs, MM_F32, mode, s);
  if (st != MM_OK) return st;
  {
    TraceScope ts("cplx_combine", s);
    cplx_combine_kernel<<<grid_for((int64_t)nc), 256, 0, s>>>(pr[0], pr[1], pr[2], pr[3],
                                                              static_cast<float2 *>(C),
                                                              (int64_t)nc);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return note_cuda(e);
  return check_device_flag(s);
}

}  // extern "C"

namespace mm {
namespace {

mm_status check_add_args(int64_t n, int64_t p, const void *A, const void *B, const void *C,
                         mm_dtype dt) {
  if (!g_ctx.inited) return MM_ENOTINIT;
  if (g_ctx.sticky) return MM_ECUDA;
  if (n < 0 || p < 0 || (dt != MM_F32 && dt != MM_F64)) return MM_EINVAL;
  if (n == 0 || p == 0) return MM_OK;
  if (!A || !B || !C || pointer_kind(A) != 1 || pointer_kind(B) != 1 || pointer_kind(C) != 1)
    return MM_EINVAL;
  return MM_EPENDING;  // valid and non-empty: queue the kernel
}

}  // namespace

mm_status enqueue_add(int64_t n, int64_t p, double alpha, const void *A, double beta,
                      const void *B, void *C, mm_dtype dt, cudaStream_t s) {
  const int64_t count = n * p;
  const bool unit = alpha == 1.0 && (beta == 1.0 || beta == -1.0);
  TraceScope ts("add", s);
  if (dt == MM_F32) {
    const bool vec = ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B) |
                       reinterpret_cast<uintptr_t>(C)) & 15) == 0 && count % 4 == 0;
    if (vec)
      add4_kernel<<<(unsigned)grid_ew(count / 4), kEwThreads, 0, s>>>(
          static_cast<const float4 *>(A), static_cast<const float4 *>(B), static_cast<float4 *>(C),
          (float)alpha, (float)beta, count / 4, unit);
    else
      add_kernel<float><<<grid_for(count), 256, 0, s>>>(
          static_cast<const float *>(A), static_cast<const float *>(B), static_cast<float *>(C),
          (float)alpha, (float)beta, count, unit);
  } else {
    add_kernel<double><<<grid_for(count), 256, 0, s>>>(
        static_cast<const double *>(A), static_cast<const double *>(B), static_cast<double *>(C),
        alpha, beta, count, unit);
  }
  return note_cuda(cudaGetLastError());
}

namespace {

}  // namespace

mm_status enqueue_scale(int64_t count, double beta, const void *D, void *C, mm_dtype dt,
                        cudaStream_t s) {
  if (count <= 0) return MM_OK;
  const size_t es = dt == MM_F64 ? 8 : 4;
  if (dt == MM_F32 ? (float)beta == 0.0f : beta == 0.0)
    return note_cuda(cudaMemsetAsync(C, 0, (size_t)count * es, s));
  TraceScope ts("add", s);
  if (dt == MM_F32)
    scale_kernel<float><<<grid_for(count), 256, 0, s>>>(static_cast<const float *>(D),
                                                        static_cast<float *>(C), (float)beta, count);
  else
    scale_kernel<double><<<grid_for(count), 256, 0, s>>>(static_cast<const double *>(D),
                                                         static_cast<double *>(C), beta, count);
  return note_cuda(cudaGetLastError());
}

namespace {

mm_status check_diag_args(int64_t n, int64_t p, const void *X, const void *d, const void *C,
                          int side, mm_dtype dt) {
  if (!g_ctx.inited) return MM_ENOTINIT;
  if (g_ctx.sticky) return MM_ECUDA;
  if (n < 0 || p < 0 || (side != 0 && side != 1) || (dt != MM_F32 && dt != MM_F64))
    return MM_EINVAL;
  if (n == 0 || p == 0) return MM_OK;
  if (!X || !d || !C || pointer_kind(X) != 1 || pointer_kind(d) != 1 || pointer_kind(C) != 1)
    return MM_EINVAL;
  return MM_EPENDING;
}

mm_status enqueue_diag(int64_t n, int64_t p, const void *X, const void *d, void *C, int side,
                       mm_dtype dt, cudaStream_t s) {
  const bool vec = dt == MM_F32 && p % 4 == 0 &&
                   ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(d) |
                     reinterpret_cast<uintptr_t>(C)) & 15) == 0;
  dim3 grid((unsigned)std::min<int64_t>((p + 255) / 256, 64),
            (unsigned)std::min<int64_t>(n, 65535));
  TraceScope ts("diag", s);
  if (vec)
    diag4_kernel<<<(unsigned)grid_ew(n * (p / 4)), kEwThreads, 0, s>>>(
        static_cast<const float4 *>(X), static_cast<const float *>(d), static_cast<float4 *>(C), n,
        p / 4, side);
  else if (dt == MM_F32)
    diag_kernel<float><<<grid, 256, 0, s>>>(static_cast<const float *>(X),
                                            static_cast<const float *>(d),
                                            static_cast<float *>(C), n, p, side);
  else
    diag_kernel<double><<<grid, 256, 0, s>>>(static_cast<const double *>(X),
                                             static_cast<const double *>(d),
                                             static_cast<double *>(C), n, p, side);
  return note_cuda(cudaGetLastError());
}

}  // namespace
}  // namespace mm

extern "C" {

mm_status mm_add(int64_t n, int64_t p, double alpha, const void *A, double beta, const void *B,
                 void *C, mm_dtype dt) {
  mm_status st = check_add_args(n, p, A, B, C, dt);
  if (st != MM_EPENDING) return st;
  std::lock_guard<std::mutex> lk(g_api_mutex);
  st = enqueue_add(n, p, alpha, A, beta, B, C, dt, g_ctx.stream);
  return st != MM_OK ? st : check_device_flag(g_ctx.stream);
}

mm_status mm_add_async(int64_t n, int64_t p, double alpha, const void *A, double beta,
                       const void *B, void *C, mm_dtype dt, void *stream) {
  mm_status st = check_add_args(n, p, A, B, C, dt);
  if (st != MM_EPENDING) return st;
  std::lock_guard<std::mutex> lk(g_api_mutex);
  return enqueue_add(n, p, alpha, A, beta, B, C, dt,
                     stream ? static_cast<cudaStream_t>(stream) : g_ctx.stream);
}

mm_status mm_diag(int64_t n, int64_t p, const void *X, const void *d, void *C, int side,
                  mm_dtype dt) {
  mm_status st = check_diag_args(n, p, X, d, C, side, dt);
  if (st != MM_EPENDING) return st;
  std::lock_guard<std::mutex> lk(g_api_mutex);
  st = enqueue_diag(n, p, X, d, C, side, dt, g_ctx.stream);
  return st != MM_OK ? st : check_device_flag(g_ctx.stream);
}

mm_status mm_diag_async(int64_t n, int64_t p, const void *X, const void *d, void *C, int side,
                        mm_dtype dt, void *stream) {
  mm_status st = check_diag_args(n, p, X, d, C, side, dt);
  if (st != MM_EPENDING) return st;
  std::lock_guard<std::mutex> lk(g_api_mutex);
  return enqueue_diag(n, p, X, d, C, side, dt,
                      stream ? static_cast<cudaStream_t>(stream) : g_ctx.stream);
}

}  // extern "C"
