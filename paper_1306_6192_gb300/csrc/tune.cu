// Autotuner of the split-BF16x3 path: tile N width (bn), K depth per stage
// (bk, with its pipeline depth), raster band height (group_m) and persistent
// grid size, chosen per size bucket by timing the candidates on the device.
// Buckets are (ceil(log2 n), ceil(log2 m), ceil(log2 p)) clamped to [5, 16].
// The table persists as text, one bucket per line:
//   ln lm lp bn bk stages group_m grid [tail]
// (tail: 1 = split the last wave's tiles along K where the tail plan gains,
// 0 = never; lines without it mean 1).
#include <cstdio>
#include <map>
#include <tuple>

#include "ctx.h"

namespace mm {
namespace {

using Key = std::tuple<int, int, int>;
std::mutex g_tune_mu;
std::map<Key, TcChoice> g_table;

int log_bucket(int64_t v) {
  int l = 0;
  while (((int64_t)1 << l) < v && l < 40) l++;
  return l < 5 ? 5 : (l > 16 ? 16 : l);
}

Key key_of(int64_t n, int64_t m, int64_t p) {
  return Key{log_bucket(n), log_bucket(m), log_bucket(p)};
}

// Heuristic used where the table has no entry: the widest N tile that the
// problem fills, K depth 32 with a 4-deep ring, bands of 16 row tiles (the
// fastest of the swept configurations at 8192^3 on GB300: 602 TFLOP/s).
TcChoice heuristic(int64_t n, int64_t m, int64_t p) {
  (void)n;
  (void)m;
  TcChoice c;
  c.bn = p > 128 ? 256 : (p > 64 ? 128 : 64);
  c.bk = 32;
  c.stages = 4;
  c.group_m = 16;
  c.grid = 0;
  return c;
}

bool valid_choice(const TcChoice &c) {
  const bool bn_ok = c.bn == 64 || c.bn == 128 || c.bn == 256;
  const bool bk_ok = (c.bk == 64 && c.stages == 2) || (c.bk == 32 && (c.stages == 3 || c.stages == 4));
  return bn_ok && bk_ok && c.group_m >= 1 && c.group_m <= 64 && c.grid >= 0 &&
         (c.tail == 0 || c.tail == 1);
}

__global__ void fill_kernel(float *x, int64_t count, float v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = v * (float)((i * 2654435761u) % 1021u) / 1021.0f - 0.5f * v;
}

}  // namespace

void tune_reset_defaults() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_table.clear();
}

TcChoice tune_choose(int64_t n, int64_t m, int64_t p) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_table.find(key_of(n, m, p));
  if (it != g_table.end()) return it->second;
  return heuristic(n, m, p);
}

mm_status tune_load_file(const char *path) {
  FILE *f = std::fopen(path, "r");
  if (!f) return MM_EINVAL;
  std::map<Key, TcChoice> t;
  char line[256];
  mm_status st = MM_OK;
  while (std::fgets(line, sizeof line, f)) {
    if (line[0] == '#' || line[0] == '\n') continue;
    int ln, lm, lp;
    TcChoice c;
    c.tail = 1;
    const int got = std::sscanf(line, "%d %d %d %d %d %d %d %d %d", &ln, &lm, &lp, &c.bn, &c.bk,
                                &c.stages, &c.group_m, &c.grid, &c.tail);
    if ((got != 8 && got != 9) || !valid_choice(c)) {
      st = MM_EINVAL;
      break;
    }
    t[Key{ln, lm, lp}] = c;
  }
  std::fclose(f);
  if (st != MM_OK) return st;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (auto &kv : t) g_table[kv.first] = kv.second;
  return MM_OK;
}

}  // namespace mm

using namespace mm;

extern "C" {

mm_status mm_tune_save(const char *path) {
  if (!path) return MM_EINVAL;
  FILE *f = std::fopen(path, "w");
  if (!f) return MM_EINVAL;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  std::fprintf(f, "# ln lm lp bn bk stages group_m grid tail\n");
  for (auto &kv : g_table) {
    const TcChoice &c = kv.second;
    std::fprintf(f, "%d %d %d %d %d %d %d %d %d\n", std::get<0>(kv.first), std::get<1>(kv.first),
                 std::get<2>(kv.first), c.bn, c.bk, c.stages, c.group_m, c.grid, c.tail);
  }
  std::fclose(f);
  return MM_OK;
}

mm_status mm_tune_load(const char *path) {
  if (!path) return MM_EINVAL;
  return tune_load_file(path);
}

mm_status mm_tune_query(int64_t n, int64_t m, int64_t p, int *bn, int *bk, int *stages,
                        int *group_m) {
  if (n < 0 || m < 0 || p < 0) return MM_EINVAL;
  TcChoice c = tune_choose(n, m, p);
  if (bn) *bn = c.bn;
  if (bk) *bk = c.bk;
  if (stages) *stages = c.stages;
  if (group_m) *group_m = c.group_m;
  return MM_OK;
}

mm_status mm_tune(int64_t n, int64_t m, int64_t p, int reps) {
  if (!g_ctx.inited) return MM_ENOTINIT;
  if (g_ctx.sticky) return MM_ECUDA;
  if (n <= 0 || m <= 0 || p <= 0 || reps <= 0) return MM_EINVAL;
  std::lock_guard<std::mutex> lk(g_api_mutex);
  cudaStream_t s = g_ctx.stream;
  float *buf = nullptr;
  const size_t ea = (size_t)(n * m), eb = (size_t)(m * p), ec = (size_t)(n * p);
  cudaError_t e = cudaMalloc(&buf, (ea + eb + ec) * sizeof(float));
  if (e != cudaSuccess) return from_cuda(e);
  fill_kernel<<<sm_count() * 4, 256, 0, s>>>(buf, (int64_t)(ea + eb), 1.0f);
  mm_problem q{n, m, p, buf, buf + ea, buf + ea + eb};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  TcChoice best{};
  float best_ms = 1e30f;
  const int bns[] = {64, 128, 256};
  const int bks[][2] = {{32, 4}, {64, 2}};
  const int gms[] = {4, 8, 16};
  mm_status st = MM_OK;
  for (int bn : bns) {
    if (bn == 64 && p > 128) continue;
    if (bn == 256 && p <= 128) continue;
    for (auto &kb : bks)
      for (int gm : gms)
      for (int tail = 1; tail >= 0; tail--) {
        TcChoice c{bn, kb[0], kb[1], gm, 0, tail};
        st = run_split(g_ctx.split_ws, &q, 1, s, &c);  // warm-up
        if (st != MM_OK) break;
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && st == MM_OK; r++) st = run_split(g_ctx.split_ws, &q, 1, s, &c);
        cudaEventRecord(e1, s);
        if (st != MM_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
          st = MM_ECUDA;
          break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
          best_ms = ms;
          best = c;
        }
      }
    if (st != MM_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  cudaFree(buf);
  if (st != MM_OK) return st;
  st = check_device_flag(s);
  if (st != MM_OK) return st;
  std::lock_guard<std::mutex> lk2(g_tune_mu);
  g_table[key_of(n, m, p)] = best;
  return MM_OK;
}

}  // extern "C"
