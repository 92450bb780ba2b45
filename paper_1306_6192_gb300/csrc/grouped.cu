// Grouped GEMM: many independent products C_g = A_g.B_g in one launch per
// kernel.  The split path puts every problem in one table (one scale launch,
// one pack launch, one persistent tensor-core launch); the SIMT FP32 and FP64
// paths use a table with a tile prefix and one block per output tile.
#include <cstring>

#include "ctx.h"

namespace mm {

mm_status enqueue_grouped(Scratch &split_ws, Scratch &tab_ws, int count, const mm_problem *probs,
                          mm_dtype dt, mm_mode mode, cudaStream_t s) {
  if (count == 0) return MM_OK;
  if (mode == MM_MODE_SPLIT_BF16X3) return run_split(split_ws, probs, count, s, nullptr);
  if (mode == MM_MODE_SPLIT_BF16X6) return run_split(split_ws, probs, count, s, nullptr, true);
  if (mode == MM_MODE_FP8) return run_fp8(g_ctx.fp8_ws, probs, count, s);
  if (mode == MM_MODE_OZAKI) {  // one emulated product after the other
    for (int g = 0; g < count; g++) {
      const mm_problem &q = probs[g];
      const mm_status st = run_ozaki(g_ctx.ozaki_ws, q.n, q.m, q.p, static_cast<const double *>(q.A),
                                     static_cast<const double *>(q.B), static_cast<double *>(q.C),
                                     g_ctx.ozaki_slices, g_ctx.ozaki_gate != 0, s);
      if (st != MM_OK) return st;
    }
    return MM_OK;
  }
  const bool f64 = dt == MM_F64;
  const int bm = f64 ? kSimtF64BM : kSimtF32BM, bn = f64 ? kSimtF64BN : kSimtF32BN;
  const int w = f64 ? 2 : 4;
  const size_t es = f64 ? 8 : 4;
  std::vector<SimtProb> tab;
  tab.reserve(count);
  int64_t tiles = 0;
  bool all_vec = true;
  for (int g = 0; g < count; g++) {
    const mm_problem &q = probs[g];
    if (q.n == 0 || q.p == 0) continue;
    if (q.m == 0) {
      cudaError_t e = cudaMemsetAsync(q.C, 0, (size_t)(q.n * q.p) * es, s);
      if (e != cudaSuccess) return from_cuda(e);
      continue;
    }
    SimtProb sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.A = q.A;
    sp.B = q.B;
    sp.C = q.C;
    sp.n = q.n;
    sp.m = q.m;
    sp.p = q.p;
    sp.tiles_n = (int32_t)ceil_div(q.p, bn);
    sp.tile_start = (int32_t)tiles;
    tiles += ceil_div(q.n, bm) * sp.tiles_n;
    auto al = [](const void *x) { return (reinterpret_cast<uintptr_t>(x) & 15) == 0; };
    all_vec = all_vec && al(q.A) && al(q.B) && al(q.C) && q.m % w == 0 && q.p % w == 0;
    tab.push_back(sp);
  }
  if (tab.empty()) return MM_OK;
  if (tiles > 0x7fffffffLL) return MM_EINVAL;
  cudaError_t e = tab_ws.reserve(tab.size() * sizeof(SimtProb), s);
  if (e != cudaSuccess) return from_cuda(e);
  e = tab_ws.stage.copy_to_device(tab_ws.ptr, tab.data(), tab.size() * sizeof(SimtProb), s);
  if (e != cudaSuccess) return from_cuda(e);
  e = launch_simt_grouped(f64, static_cast<const SimtProb *>(tab_ws.ptr), (int)tab.size(),
                          (int)tiles, all_vec, s);
  return from_cuda(e);
}

}  // namespace mm
