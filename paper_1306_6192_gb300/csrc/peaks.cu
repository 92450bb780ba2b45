// Measured FMA throughput of the CUDA cores (FP32 FFMA, FP64 DFMA): the
// denominators of the SIMT FP32 and FP64 DGEMM kernels' rooflines.  A grid of
// several blocks per SM runs independent FMA chains on registers for a fixed
// number of iterations; the rate is the FMAs executed (2 flops each) over the
// kernel's CUDA-event time.  The multiplier and addend are loaded from device
// memory into per-thread registers (two copies, picked by the thread index,
// so the compiler cannot keep them in uniform registers): as kernel
// parameters (constant-bank operands) the FP64 FMAs issued ~17 % slower on
// the GB300 (1.008 against 1.207 TFLOP/s), below the rate the DGEMM kernel
// itself reaches.  It only reads the device;
// nothing about the device's clocks or settings is changed.  Not part of the
// paper.
#include <cuda_runtime.h>

#include "ctx.h"

namespace mm {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kChains = 12;  // independent FMA chains per thread

template <typename T>
__global__ void __launch_bounds__(kPeakThreads)
fma_peak_kernel(int64_t iters, T *buf) {
  const T a = buf[1 + (threadIdx.x & 1)], b = buf[3 + (threadIdx.x & 1)];  // per-thread registers
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; c++) x[c] = (T)(threadIdx.x + c) * (T)1e-7;
  for (int64_t i = 0; i < iters; i++) {
#pragma unroll
    for (int r = 0; r < 16; r++) {
#pragma unroll
      for (int c = 0; c < kChains; c++) x[c] = fma(x[c], a, b);
    }
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; c++) s += x[c];
  if (s == (T)12345.678) buf[0] = s;  // keeps the chains live; never true in practice
}

template <typename T>
cudaError_t measure(int64_t iters, double *flops_per_s, cudaStream_t st) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_peak_kernel<T>, kPeakThreads, 0);
  if (e != cudaSuccess) return e;
  const int blocks = sms * (per_sm > 0 ? per_sm : 1);
  T *buf = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  // the result slot, then a multiplier just below 1 and a tiny addend (the
  // values stay finite and normal)
  const T host[5] = {(T)0, (T)0.999999, (T)0.999999, (T)1e-9, (T)1e-9};
  e = cudaMalloc(&buf, sizeof(host));
  if (e == cudaSuccess) e = cudaMemcpyAsync(buf, host, sizeof(host), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    fma_peak_kernel<T><<<blocks, kPeakThreads, 0, st>>>(iters / 8 + 1, buf);
    e = cudaEventRecord(e0, st);
  }
  if (e == cudaSuccess) {
    fma_peak_kernel<T><<<blocks, kPeakThreads, 0, st>>>(iters, buf);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess && ms > 0.0f)
    *flops_per_s = 2.0 * (double)blocks * kPeakThreads * kChains * 16.0 * (double)iters /
                   ((double)ms * 1e-3);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (buf) {
    cudaStreamSynchronize(st);  // the kernels are done with it
    cudaFree(buf);
  }
  return e;
}

}  // namespace
}  // namespace mm

using namespace mm;

extern "C" mm_status mm_measure_fma_peak(mm_dtype dt, int64_t iters, double *flops_per_s) {
  if (!g_ctx.inited) return MM_ENOTINIT;
  if (g_ctx.sticky) return MM_ECUDA;
  if (!flops_per_s || iters < 1 || (dt != MM_F32 && dt != MM_F64)) return MM_EINVAL;
  std::lock_guard<std::mutex> lk(g_api_mutex);
  *flops_per_s = 0.0;
  const cudaError_t e = dt == MM_F64 ? measure<double>(iters, flops_per_s, g_ctx.stream)
                                     : measure<float>(iters, flops_per_s, g_ctx.stream);
  return note_cuda(e);
}
