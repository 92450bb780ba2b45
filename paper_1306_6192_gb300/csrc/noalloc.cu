// FP32 split-BF16 product that allocates nothing: the scratch of the split
// path (scale words, problem table, packed bf16 operands and the device
// timeout flag) lives in one fixed file-scope device array instead of
// library buffers obtained with cudaMalloc.
//
// Who needs it: callers that must not allocate device memory - a plug-in
// running inside a host framework that owns and accounts for all device
// memory, code on a latency-critical path that cannot afford cudaMalloc's
// implicit synchronisation, a process whose memory budget is fixed at
// start-up.  Such a caller passes its own A, B and C and gets the same
// kernels and tile choices as mm_gemm's split path.
//
// Limits and sharing rules:
//   - kNoAllocBytes (64 MiB) bounds a problem's scratch: products whose packed
//     operands do not fit are rejected with MM_ESCRATCH (about 2048^3 fits,
//     3072^3 does not).  Every GPU that loads the library holds this array
//     until the process exits.
//   - All calls share the one array: calls whose work overlaps on the GPU
//     (different streams, or different host threads on one device) race and
//     corrupt each other's results.  Serialise them.
//   - The first call on a device looks up the array's device address there
//     (cudaGetSymbolAddress, with that device current); make that first call
//     before any stream capture.
//   - Every call waits for its stream before it returns: it reads the device
//     timeout flag back to report MM_ETIMEOUT.
//   - The split path's other kernels are reused unchanged; nothing here
//     depends on mm_init.
// There is no counterpart in the paper.
#include <cstring>

#include "ctx.h"

namespace mm {
namespace {

constexpr size_t kNoAllocBytes = (size_t)64 << 20;
constexpr size_t kFlagOff = 0;      // int timeout flag
constexpr size_t kScaleFlagOff = 64;  // int per-operand scale flags
constexpr size_t kTableOff = 256;   // one SplitProb
constexpr size_t kScalesOff = 512;  // uint32 per row of A and column of B
static_assert(sizeof(SplitProb) <= kScalesOff - kTableOff, "table slot");
constexpr int kMaxDevices = 64;

static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocBytes];

std::mutex g_setup_mu;
void *g_scratch_addr[kMaxDevices];
int g_sms[kMaxDevices];

// Per-device set-up: the array's device address (host code cannot use the
// symbol itself) and the SM count, with `dev` current.
mm_status setup(int dev, void **addr, int *sms) {
  if (dev < 0 || dev >= kMaxDevices) return MM_EUNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    int major = 0, minor = 0, count = 0;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return MM_ECUDA;
    if (major != 10 || minor != 3) return MM_EUNSUPPORTED;
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return MM_ECUDA;
    }
    g_sms[dev] = count;
    g_scratch_addr[dev] = p;
  }
  *addr = g_scratch_addr[dev];
  *sms = g_sms[dev];
  return MM_OK;
}

}  // namespace
}  // namespace mm

using namespace mm;

extern "C" {

mm_status mm_gemm_split_static(int64_t n, int64_t m, int64_t p, const float *A, const float *B,
                               float *C, void *stream) {
  if (n < 0 || m < 0 || p < 0) return MM_EINVAL;
  if (n == 0 || p == 0) return MM_OK;
  if (!C || (m > 0 && (!A || !B))) return MM_EINVAL;
  if (n > ((int64_t)1 << 31) || m > ((int64_t)1 << 31) || p > ((int64_t)1 << 31))
    return MM_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MM_ECUDA;
  void *addr = nullptr;
  int sms = 0;
  mm_status st = setup(dev, &addr, &sms);
  if (st != MM_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint8_t *base = static_cast<uint8_t *>(addr);
  if (m == 0) {
    if (cudaMemsetAsync(C, 0, (size_t)(n * p) * sizeof(float), s) != cudaSuccess) return MM_ECUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? MM_OK : MM_ECUDA;
  }
  // Same tile choice and split kind as mm_gemm's split path for this size.
  TcChoice ch = tune_choose(n, m, p);
  const TcKind kind = split_kind_for(m);
  ch.bn = tc_bn(kind, ch.bn);
  const int parts = pack_parts(kind);
  SplitProb sp;
  std::memset(&sp, 0, sizeof(sp));
  sp.A = A;
  sp.B = B;
  sp.C = C;
  sp.n = (int32_t)n;
  sp.m = (int32_t)m;
  sp.p = (int32_t)p;
  sp.bn = ch.bn;
  sp.group_m = ch.group_m;
  sp.mt = (int32_t)ceil_div(n, kTcBM);
  sp.nt = (int32_t)ceil_div(p, ch.bn);
  sp.kt = (int32_t)ceil_div(m, pack_k(kind));
  const int64_t a_rows = (int64_t)sp.mt * sp.kt * parts * kTcBM;
  const int64_t rows = a_rows + (int64_t)sp.nt * sp.kt * parts * ch.bn;
  const size_t part_off = (kScalesOff + (size_t)(n + p) * 4 + 255) & ~(size_t)255;
  const size_t pack_off = (part_off + (size_t)sp.kt * (n + p) * 4 + 1023) & ~(size_t)1023;
  if (pack_off + (size_t)rows * kPackRowBytes > kNoAllocBytes) return MM_ESCRATCH;
  uint8_t *pack = base + pack_off;
  sp.a_row0 = 0;
  sp.b_row0 = a_rows;
  sp.sA = reinterpret_cast<uint32_t *>(base + kScalesOff);
  sp.tB = sp.sA + n;
  sp.pA = reinterpret_cast<uint32_t *>(base + part_off);
  sp.pB = sp.pA + (int64_t)sp.kt * n;
  sp.unit_start = 0;  // no tail split: split_s = 0 from the memset
  sp.pack_start = 0;
  const int64_t tiles = (int64_t)sp.mt * sp.nt;
  const int64_t packs = (int64_t)sp.mt * sp.kt + (int64_t)sp.nt * sp.kt;
  SplitProb *d_tab = reinterpret_cast<SplitProb *>(base + kTableOff);
  int *d_flag = reinterpret_cast<int *>(base + kFlagOff);
  // The array keeps the previous call's contents: the timeout and scale flags
  // must start at zero; the maxima and every pack row the kernels read are
  // rewritten (zero padding included) by the pack and verify kernels.
  cudaError_t e = cudaMemsetAsync(d_flag, 0, 128, s);  // timeout flag and scale flags
  if (e == cudaSuccess) e = cudaMemsetAsync(sp.sA, 0, (size_t)(n + p) * 4, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_tab, &sp, sizeof(sp), cudaMemcpyHostToDevice, s);
  int *d_sflag = reinterpret_cast<int *>(base + kScaleFlagOff);
  // same passes as mm_gemm's split path: unscaled pack with the maxima,
  // verification, re-pack of operands out of range
  if (e == cudaSuccess)
    e = launch_split_pack(kind, kPackUnscaled, d_tab, 1, (int)packs, nullptr, nullptr, nullptr,
                          pack, s);
  // d_sflag[0]: the operands' scale flags; d_sflag[1]: set when any is flagged
  if (e == cudaSuccess)
    e = launch_split_verify(d_tab, 1, verify_items(n, p), nullptr, d_sflag, d_sflag + 1, sp.kt,
                            s);
  if (e == cudaSuccess)
    e = launch_split_pack(kind, kPackFix, d_tab, 1, (int)packs, nullptr, d_sflag, d_sflag + 1,
                          pack, s);
  if (e == cudaSuccess) {
    // the tuned grid (0: one CTA per SM of this device, counted at set-up)
    const int grid = ch.grid > 0 ? ch.grid : sms;
    TcConfig cfg = kind == kTcSplitBf16x3 ? TcConfig{2 * ch.bk, ch.stages, grid, ch.bn}
                                          : TcConfig{64, 3, grid, ch.bn};
    e = launch_tc(kind, d_tab, 1, (int)tiles, nullptr, d_sflag, pack, rows, cfg, d_flag, s);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorInvalidValue ? MM_EINVAL : MM_ECUDA;
  }
  int flag = 0;
  e = cudaMemcpyAsync(&flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return MM_ECUDA;
  return flag != 0 ? MM_ETIMEOUT : MM_OK;
}

}  // extern "C"
