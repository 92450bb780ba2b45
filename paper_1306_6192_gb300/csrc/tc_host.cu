// Host side of the packed split path (split-BF16x3 / x6): builds the problem
// tables, lays out the scratch (pack rows, scale words, tables) and queues
// prep + tensor-core kernels, one launch per kernel and kind; and the fused
// split-K path's plan and launch.
#include <cmath>
#include <cstring>

#include "ctx.h"

namespace mm {

TcKind split_kind_for(int64_t m) {
  return 3.1 * std::ldexp(1.0, -16) <= 1e-6 * std::sqrt((double)m) ? kTcSplitBf16x3
                                                                    : kTcSplitBf16x6;
}

namespace {

struct Group {
  TcKind kind;
  TcConfig cfg{0, 0, 0};
  std::vector<SplitProb> tab;
  int64_t units = 0, packs = 0;  // tensor-core work units, pack tiles
  int64_t vers = 0;               // verify items
  int max_kt = 0;                           // longest K (pack rows) of the table
};

double kind_products(TcKind k) {
  return k == kTcSplitBf16x3 ? 3.0 : (k == kTcSplitBf16x6 ? 6.0 : 0.5);
}

// Tail split of one product from its own shape and tile choice; fills
// split_from / split_s and returns the plan.
TcTail plan_tail(SplitProb &sp, TcKind kind, const TcChoice &ch) {
  const TcConfig cfg{0, 0, ch.grid};
  TcTail t = ch.tail ? tc_tail_plan((int64_t)sp.mt * sp.nt, tc_grid(cfg), sp.kt, sp.bn, sp.m,
                                    kind_products(kind))
                     : TcTail{sp.mt * sp.nt, 1};
  sp.split_from = t.split_from;
  sp.split_s = t.split_s;
  return t;
}

mm_status run_tc_groups(Scratch &ws, const mm_problem *probs, int count, cudaStream_t s,
                        const TcChoice *force, bool six, const Epi *epi) {
  Group groups[2] = {{kTcSplitBf16x3}, {kTcSplitBf16x6}};
  int64_t rows = 0, scal = 0, part = 0;
  size_t tail_parts = 0, tail_cnts = 0;  // partial tiles and counters of tail splits
  for (int g = 0; g < count; g++) {
    const mm_problem &q = probs[g];
    if (q.n == 0 || q.p == 0) continue;
    if (q.m == 0) {
      cudaError_t e = cudaMemsetAsync(q.C, 0, (size_t)(q.n * q.p) * sizeof(float), s);
      if (e != cudaSuccess) return note_cuda(e);
      continue;
    }
    const TcKind kind = six ? kTcSplitBf16x6 : split_kind_for(q.m);
    Group &G = groups[kind == kTcSplitBf16x3 ? 0 : 1];
    TcChoice ch = force ? *force : tune_choose(q.n, q.m, q.p);
    ch.bn = tc_bn(kind, ch.bn);
    if (G.tab.empty()) {
      if (kind == kTcSplitBf16x3) G.cfg = TcConfig{2 * ch.bk, ch.stages, ch.grid};
      else G.cfg = TcConfig{64, 3, ch.grid};
    }
    const int parts = pack_parts(kind);
    SplitProb sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.A = static_cast<const float *>(q.A);
    sp.B = static_cast<const float *>(q.B);
    sp.C = static_cast<float *>(q.C);
    if (epi && count == 1) sp.epi = epi->as<float>();
    sp.n = (int32_t)q.n;
    sp.m = (int32_t)q.m;
    sp.p = (int32_t)q.p;
    sp.bn = ch.bn;
    sp.group_m = ch.group_m;
    sp.mt = (int32_t)ceil_div(q.n, kTcBM);
    sp.nt = (int32_t)ceil_div(q.p, ch.bn);
    sp.kt = (int32_t)ceil_div(q.m, pack_k(kind));
    sp.a_row0 = rows;
    rows += (int64_t)sp.mt * sp.kt * parts * kTcBM;
    sp.b_row0 = rows;
    rows += (int64_t)sp.nt * sp.kt * parts * ch.bn;
    sp.sA = reinterpret_cast<uint32_t *>((uintptr_t)scal);  // offsets, fixed below
    scal += q.n;
    sp.tB = reinterpret_cast<uint32_t *>((uintptr_t)scal);
    scal += q.p;
    // partial maxima of the unscaled pack
    sp.pA = reinterpret_cast<uint32_t *>((uintptr_t)part);
    part += (int64_t)sp.kt * q.n;
    sp.pB = reinterpret_cast<uint32_t *>((uintptr_t)part);
    part += (int64_t)sp.kt * q.p;
    sp.ver_start = (int32_t)G.vers;
    G.vers += verify_items(q.n, q.p);
    G.max_kt = std::max(G.max_kt, sp.kt);
    const TcTail tail = plan_tail(sp, kind, ch);
    if (tail.split_s > 1) {  // offsets, fixed below
      sp.part = reinterpret_cast<float *>((uintptr_t)tail_parts);
      sp.cnt = reinterpret_cast<int *>((uintptr_t)tail_cnts);
      tail_parts += tc_tail_part_bytes(tail, (int64_t)sp.mt * sp.nt, sp.bn);
      tail_cnts += (size_t)((int64_t)sp.mt * sp.nt - tail.split_from);
    }
    sp.unit_start = (int32_t)G.units;
    G.units += split_units(sp);
    G.cfg.max_bn = G.tab.empty() ? sp.bn : std::max(G.cfg.max_bn, sp.bn);
    sp.pack_start = (int32_t)G.packs;
    G.packs += (int64_t)sp.mt * sp.kt + (int64_t)sp.nt * sp.kt;
    G.tab.push_back(sp);
  }
  size_t ntab = 0;
  for (auto &G : groups) {
    if (G.units > 0x7fffffffLL || G.packs > 0x7fffffffLL || G.vers > 0x7fffffffLL)
      return MM_EINVAL;
    ntab += G.tab.size();
  }
  if (ntab == 0) return MM_OK;
  if (rows > 0x7fffffffLL) return MM_EINVAL;
  // Layout: packs | the words that start at zero (scale words, per-problem
  // scale flags and one "any flagged" word per group, tail-split counters: one
  // memset clears them) | partial maxima | table | item maps | partial tiles
  const size_t pack_bytes = (size_t)rows * kPackRowBytes;
  const size_t scal_off = (pack_bytes + 255) & ~(size_t)255;
  const size_t flag_off = scal_off + (size_t)scal * 4;
  const size_t tcnt_off = flag_off + (ntab + 3) * sizeof(int);
  const size_t zero_end = tcnt_off + tail_cnts * sizeof(int);
  const size_t part_off = (zero_end + 255) & ~(size_t)255;
  const size_t tab_off = (part_off + (size_t)part * 4 + 255) & ~(size_t)255;
  // item -> problem maps (work units, pack tiles and verify items) of each
  // group with more than one problem
  size_t map_ints = 0;
  for (auto &G : groups)
    if (G.tab.size() > 1) map_ints += (size_t)(G.units + G.packs + G.vers);
  // the work units of each CTA for groups of several problems (their units
  // differ in length), written with the table in one copy
  std::vector<int> orders[2];
  size_t order_ints = 0;
  for (int gi = 0; gi < 2; gi++) {
    Group &G = groups[gi];
    if (G.tab.size() <= 1) continue;
    tc_unit_order(G.tab.data(), (int)G.tab.size(), tc_launch_grid(G.cfg, G.units), orders[gi]);
    order_ints += orders[gi].size();
  }
  const size_t tab_bytes = (ntab * sizeof(SplitProb) + 15) & ~(size_t)15;
  // tensor maps over the C matrices for the epilogue's tiled stores, for
  // tables of up to kMaxCMaps products (each map is encoded on the host)
  constexpr size_t kMaxCMaps = 8192, kMapBytes = 128;
  const size_t cmap_rel = (tab_bytes + order_ints * sizeof(int) + 63) & ~(size_t)63;
  const size_t cmap_bytes = ntab <= kMaxCMaps ? ntab * kMapBytes : 0;
  const size_t map_off = (tab_off + cmap_rel + cmap_bytes + 255) & ~(size_t)255;
  const size_t tpart_off = (map_off + map_ints * sizeof(int) + 255) & ~(size_t)255;
  const size_t need = tpart_off + tail_parts;
  cudaError_t e = ws.reserve(need, s);
  if (e != cudaSuccess) return note_cuda(e);
  uint8_t *base = static_cast<uint8_t *>(ws.ptr);
  std::vector<SplitProb> all;
  all.reserve(ntab);
  for (auto &G : groups)
    for (auto &sp : G.tab) {
      sp.sA = reinterpret_cast<uint32_t *>(base + scal_off) + (uintptr_t)sp.sA;
      sp.tB = reinterpret_cast<uint32_t *>(base + scal_off) + (uintptr_t)sp.tB;
      sp.pA = reinterpret_cast<uint32_t *>(base + part_off) + (uintptr_t)sp.pA;
      sp.pB = reinterpret_cast<uint32_t *>(base + part_off) + (uintptr_t)sp.pB;
      if (sp.split_s > 1) {
        sp.part = reinterpret_cast<float *>(base + tpart_off + (uintptr_t)sp.part);
        sp.cnt = reinterpret_cast<int *>(base + tcnt_off) + (uintptr_t)sp.cnt;
      }
      all.push_back(sp);
    }
  SplitProb *d_tab = reinterpret_cast<SplitProb *>(base + tab_off);
  int *d_orders = reinterpret_cast<int *>(base + tab_off + tab_bytes);
  const void *d_cmaps = cmap_bytes ? static_cast<const void *>(base + tab_off + cmap_rel) : nullptr;
  {
    // one copy: the table, the CTAs' unit lists, the C tensor maps
    std::vector<uint8_t> blob(cmap_rel + cmap_bytes, 0);
    for (size_t k = 0; cmap_bytes && k < ntab; k++) {
      SplitProb &sp = all[k];
      // the epilogue C = alpha (A.B) + beta D loads D in 16-byte vectors
      // beside the tiled stores (a D off that alignment: plain stores)
      const bool d_ok = sp.epi.on != 2 || (reinterpret_cast<uintptr_t>(sp.epi.D) & 15u) == 0;
      if (d_ok && tc_c_map_ok(sp.C, sp.n, sp.p) &&
          encode_c_map(blob.data() + cmap_rel + k * kMapBytes, sp.C, sp.n, sp.p) == cudaSuccess)
        sp.c_tma = (int32_t)k + 1;
    }
    std::memcpy(blob.data(), all.data(), all.size() * sizeof(SplitProb));
    size_t at = tab_bytes;
    for (auto &o : orders) {
      if (o.empty()) continue;
      std::memcpy(blob.data() + at, o.data(), o.size() * sizeof(int));
      at += o.size() * sizeof(int);
    }
    e = ws.stage.copy_to_device(d_tab, blob.data(), blob.size(), s);
  }
  if (e != cudaSuccess) return note_cuda(e);
  e = cudaMemsetAsync(base + scal_off, 0, zero_end - scal_off, s);
  if (e != cudaSuccess) return note_cuda(e);
  size_t off = 0;
  int *flags_all = reinterpret_cast<int *>(base + flag_off);
  int *maps = reinterpret_cast<int *>(base + map_off);
  for (int gi = 0; gi < 2; gi++) {
    Group &G = groups[gi];
    if (G.tab.empty()) continue;
    const SplitProb *dt = d_tab + off;
    int *flags = flags_all + off;
    int *any = flags_all + ntab + gi;
    const int np = (int)G.tab.size();
    off += G.tab.size();
    int *tile_map = nullptr, *pack_map = nullptr, *ver_map = nullptr;
    const int *order = nullptr;
    if (!orders[gi].empty()) {
      order = d_orders;
      d_orders += orders[gi].size();
    }
    if (np > 1) {
      tile_map = maps;
      pack_map = tile_map + G.units;
      ver_map = pack_map + G.packs;
      maps = ver_map + G.vers;
      e = launch_split_maps(dt, np, tile_map, pack_map, ver_map, s);
      if (e != cudaSuccess) return note_cuda(e);
    }
    // one unscaled pass that also reduces the maxima, then the operands out
    // of range are re-packed with their scales
    e = launch_split_pack(G.kind, kPackUnscaled, dt, np, (int)G.packs, pack_map, nullptr, nullptr,
                          base, s);
    if (e == cudaSuccess) e = launch_split_verify(dt, np, G.vers, ver_map, flags, any, G.max_kt, s);
    if (e == cudaSuccess)
      e = launch_split_pack(G.kind, kPackFix, dt, np, (int)G.packs, pack_map, flags, any, base, s);
    if (e == cudaSuccess)
      e = launch_tc(G.kind, dt, np, (int)G.units, tile_map, flags, base, rows, G.cfg, g_ctx.d_err,
                    s, order, 0, d_cmaps);
    if (e != cudaSuccess) return note_cuda(e);
  }
  return MM_OK;
}

}  // namespace

mm_status run_split_chunked(Scratch &ws, int64_t n, int64_t m, int64_t p, const float *A,
                            const float *B, float *C, int chunks, const int64_t *row0,
                            cudaStream_t s, cudaEvent_t *in_ready, cudaEvent_t *out_ready) {
  if (n == 0 || p == 0) return MM_OK;
  const TcKind kind = split_kind_for(m);
  const int parts = pack_parts(kind);
  TcChoice ch = tune_choose(n, m, p);
  ch.bn = tc_bn(kind, ch.bn);
  const TcConfig cfg = kind == kTcSplitBf16x3 ? TcConfig{2 * ch.bk, ch.stages, ch.grid, ch.bn}
                                              : TcConfig{64, 3, ch.grid, ch.bn};
  const int32_t kt = (int32_t)ceil_div(m, pack_k(kind));
  const int32_t nt = (int32_t)ceil_div(p, ch.bn);
  // layout: B pack, then each slab's A pack; scale words: B columns, then A rows
  int64_t rows = (int64_t)nt * kt * parts * ch.bn;
  std::vector<SplitProb> tab((size_t)chunks);
  std::vector<int64_t> tiles((size_t)chunks), packs((size_t)chunks);
  for (int c = 0; c < chunks; c++) {
    const int64_t r0 = row0[c], r1 = row0[c + 1];
    SplitProb &sp = tab[(size_t)c];
    std::memset(&sp, 0, sizeof(sp));
    sp.A = A + r0 * m;
    sp.B = B;
    sp.C = C + r0 * p;
    sp.n = (int32_t)(r1 - r0);
    sp.m = (int32_t)m;
    sp.p = (int32_t)p;
    sp.bn = ch.bn;
    sp.group_m = ch.group_m;
    sp.mt = (int32_t)ceil_div(r1 - r0, kTcBM);
    sp.nt = nt;
    sp.kt = kt;
    sp.b_row0 = 0;
    sp.a_row0 = rows;
    rows += (int64_t)sp.mt * kt * parts * kTcBM;
    sp.sA = reinterpret_cast<uint32_t *>((uintptr_t)(p + r0));  // offsets, fixed below
    sp.tB = reinterpret_cast<uint32_t *>((uintptr_t)0);
    // partial maxima: B's columns first (kt * p), then each slab's rows
    sp.pA = reinterpret_cast<uint32_t *>((uintptr_t)((int64_t)kt * p + (int64_t)kt * r0));
    sp.pB = reinterpret_cast<uint32_t *>((uintptr_t)0);
    // slabs are not tail-split: each slab's last wave is filled by the next
    // slab's GEMM on the other tensor-core stream
    sp.split_s = 1;
    sp.unit_start = 0;
    tiles[(size_t)c] = (int64_t)sp.mt * nt;
    // slab 0 also scales and packs B; the other slabs reuse its pack
    packs[(size_t)c] = (int64_t)sp.mt * kt + (c == 0 ? (int64_t)nt * kt : 0);
  }
  if (rows > 0x7fffffffLL) return MM_EINVAL;
  const size_t pack_bytes = (size_t)rows * kPackRowBytes;
  const size_t scal_off = (pack_bytes + 255) & ~(size_t)255;
  const size_t part_off = (scal_off + (size_t)(n + p) * 4 + 255) & ~(size_t)255;
  const size_t tab_off = (part_off + (size_t)kt * (n + p) * 4 + 255) & ~(size_t)255;
  // per slab: its scale flags word, then (chunks words later) its "any" word
  const size_t flag_off = (tab_off + tab.size() * sizeof(SplitProb) + 255) & ~(size_t)255;
  cudaError_t e = ws.reserve(flag_off + 2 * tab.size() * sizeof(int), s);
  if (e != cudaSuccess) return note_cuda(e);
  uint8_t *base = static_cast<uint8_t *>(ws.ptr);
  uint32_t *scal = reinterpret_cast<uint32_t *>(base + scal_off);
  uint32_t *part = reinterpret_cast<uint32_t *>(base + part_off);
  for (auto &sp : tab) {
    sp.sA = scal + (uintptr_t)sp.sA;
    sp.tB = scal + (uintptr_t)sp.tB;
    sp.pA = part + (uintptr_t)sp.pA;
    sp.pB = part + (uintptr_t)sp.pB;
  }
  SplitProb *d_tab = reinterpret_cast<SplitProb *>(base + tab_off);
  e = ws.stage.copy_to_device(d_tab, tab.data(), tab.size() * sizeof(SplitProb), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(scal, 0, (size_t)(n + p) * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(base + flag_off, 0, 2 * tab.size() * sizeof(int), s);
  if (e != cudaSuccess) return note_cuda(e);
  // Preparation of the slabs runs in order on s; each slab's tensor-core
  // launch goes to one of two streams, so the next slab's preparation and
  // GEMM fill the last partial wave of the previous one.
  for (int c = 0; c < chunks; c++) {
    if (c == 0 && (e = cudaStreamWaitEvent(s, in_ready[0], 0)) != cudaSuccess) break;
    if ((e = cudaStreamWaitEvent(s, in_ready[c + 1], 0)) != cudaSuccess) break;
    const SplitProb *dt = d_tab + c;
    int *flag = reinterpret_cast<int *>(base + flag_off) + c;
    int *any = flag + chunks;
    // slab 0 packs (and reduces) B as well; a later slab's verify sees all of
    // B's column maxima, so its B flag equals slab 0's, and it leaves B's
    // column words (read by the GEMMs in flight) untouched
    if ((e = launch_split_pack(kind, kPackUnscaled, dt, 1, (int)packs[(size_t)c], nullptr, nullptr,
                               nullptr, base, s)) != cudaSuccess)
      break;
    if ((e = launch_split_verify(dt, 1, verify_items(tab[(size_t)c].n, p), nullptr, flag, any, kt,
                                 s, c == 0)) != cudaSuccess)
      break;
    if ((e = launch_split_pack(kind, kPackFix, dt, 1, (int)packs[(size_t)c], nullptr, flag, any,
                               base, s)) != cudaSuccess)
      break;
    if ((e = cudaEventRecord(g_ctx.ev_prep[c], s)) != cudaSuccess) break;
    cudaStream_t t = g_ctx.tc_streams[c & 1];
    if ((e = cudaStreamWaitEvent(t, g_ctx.ev_prep[c], 0)) != cudaSuccess) break;
    if ((e = launch_tc(kind, dt, 1, (int)tiles[(size_t)c], nullptr, flag, base, rows, cfg,
                       g_ctx.d_err, t)) != cudaSuccess)
      break;
    if ((e = cudaEventRecord(out_ready[c], t)) != cudaSuccess) break;
  }
  // s waits for every slab's GEMM: the caller's later work on s is ordered
  for (int c = 0; c < chunks && e == cudaSuccess; c++) e = cudaStreamWaitEvent(s, out_ready[c], 0);
  return note_cuda(e);
}

mm_status run_split(Scratch &ws, const mm_problem *probs, int count, cudaStream_t s,
                    const TcChoice *force, bool six, const Epi *epi) {
  return run_tc_groups(ws, probs, count, s, force, six, epi);
}

mm_status run_fp8(Scratch &ws, const mm_problem *probs, int count, cudaStream_t s) {
  return run_fp8_blocks(ws, probs, count, s);
}

}  // namespace mm

namespace mm {

TcTail product_tail(int64_t n, int64_t m, int64_t p, TcKind kind, int64_t *tiles_out) {
  TcChoice ch = tune_choose(n, m, p);
  ch.bn = tc_bn(kind, ch.bn);
  SplitProb sp;
  std::memset(&sp, 0, sizeof(sp));
  sp.n = (int32_t)n;
  sp.m = (int32_t)m;
  sp.p = (int32_t)p;
  sp.bn = ch.bn;
  sp.mt = (int32_t)ceil_div(n, kTcBM);
  sp.nt = (int32_t)ceil_div(p, ch.bn);
  sp.kt = (int32_t)ceil_div(m, pack_k(kind));
  if (tiles_out) *tiles_out = (int64_t)sp.mt * sp.nt;
  return plan_tail(sp, kind, ch);
}

size_t tail_scratch_bytes(int64_t n, int64_t m, int64_t p, TcKind kind) {
  if (n <= 0 || m <= 0 || p <= 0) return 0;
  int64_t tiles = 0;
  const TcTail t = product_tail(n, m, p, kind, &tiles);
  TcChoice ch = tune_choose(n, m, p);
  return tc_tail_bytes(t, tiles, tc_bn(kind, ch.bn));
}

}  // namespace mm

using namespace mm;

extern "C" mm_status mm_tune_query_tail(int64_t n, int64_t m, int64_t p, int *tiles,
                                        int *split_from, int *split_s) {
  if (!g_ctx.inited) return MM_ENOTINIT;
  if (n < 0 || m < 0 || p < 0) return MM_EINVAL;
  int64_t t = 0;
  TcTail tail{0, 1};
  if (n > 0 && m > 0 && p > 0) {
    const TcKind kind = split_kind_for(m);
    tail = product_tail(n, m, p, kind, &t);
    if (t > 0x7fffffffLL) return MM_EINVAL;
  }
  if (tail.split_s <= 1) tail = TcTail{(int)t, 1};
  if (tiles) *tiles = (int)t;
  if (split_from) *split_from = tail.split_from;
  if (split_s) *split_s = tail.split_s;
  return MM_OK;
}

extern "C" mm_status mm_tail_plan(int64_t tiles, int grid, int kt, int bn, int64_t m,
                                  double products, int *split_from, int *split_s) {
  if (tiles < 0 || tiles > 0x7fffffffLL || grid < 0 || kt < 0 || bn <= 0 || m < 0 ||
      !(products > 0.0) || !split_from || !split_s)
    return MM_EINVAL;
  const TcTail t = tc_tail_plan(tiles, grid, kt, bn, m, products);
  *split_from = t.split_s > 1 ? t.split_from : (int)tiles;
  *split_s = t.split_s > 1 ? t.split_s : 1;
  return MM_OK;
}

// ------------------------------------------------------ fused split-K path
namespace mm {

FusedPlan fused_plan(int64_t n, int64_t m, int64_t p, TcKind kind) {
  FusedPlan best{0, 0, 0};
  if (kind == kTcE4m3 || n <= 0 || m <= 0 || p <= 0) return best;
  const int64_t tiles = ceil_div(n, kTcBM) * ceil_div(p, 128);
  const int64_t kb = ceil_div(m, 64);
  // products that fill at least half of the SMs with whole tiles keep the
  // packed path (their operands are converted once, not once per tile)
  if (2 * tiles > sm_count()) return best;
  const bool six = kind == kTcSplitBf16x6;
  // cost in units of one K block of one CTA (its conversion dominates): the
  // blocks of the longest slice, the cluster's exchange through distributed
  // shared memory, and the clusters' meeting in global memory, whose last
  // cluster reads Q partial tiles
  double best_cost = 1e300;
  for (int cs : {8, 4, 2, 1}) {
    const int cap = fused_capacity(six, cs);
    if (cap <= 0) continue;
    for (int64_t q = 1;; q++) {
      const int64_t S = q * cs;
      if (S > kb || tiles * S > cap) break;
      const double cost = (double)ceil_div(kb, S) + (cs > 1 ? 0.3 : 0.0) +
                          (q > 1 ? 0.5 + 0.1 * (double)q : 0.0);
      if (cost < best_cost - 1e-9 || (cost < best_cost + 1e-9 && S < best.S)) {
        best_cost = cost;
        best = FusedPlan{(int)S, (int)q, cs};
      }
    }
  }
  // a slice of more than eight K blocks is slower here than on the packed
  // path, whose operands are split once and streamed by TMA (GB300, 1024^3:
  // 52 us fused at eight blocks per slice against 58 us packed; 1024 x 2048
  // x 1024 at sixteen: 90 against 69 us)
  if (best.S > 0 && ceil_div(kb, best.S) > 8) best = FusedPlan{0, 0, 0};
  return best;
}

mm_status run_fused(Scratch &ws, int64_t n, int64_t m, int64_t p, const float *A, const float *B,
                    float *C, TcKind kind, const FusedPlan &plan, cudaStream_t s,
                    const Epi *epi) {
  FusedProb fp;
  std::memset(&fp, 0, sizeof(fp));
  fp.A = A;
  fp.B = B;
  fp.C = C;
  fp.epi = epi_of<float>(epi);
  fp.n = (int32_t)n;
  fp.m = (int32_t)m;
  fp.p = (int32_t)p;
  fp.mt = (int32_t)ceil_div(n, kTcBM);
  fp.nt = (int32_t)ceil_div(p, 128);
  fp.kb = (int32_t)ceil_div(m, 64);
  fp.S = plan.S;
  fp.Q = plan.Q;
  const int64_t tiles = (int64_t)fp.mt * fp.nt;
  cudaError_t e = cudaSuccess;
  if (plan.Q > 1) {
    // counters first (kept at zero between launches: the last cluster of a
    // chunk resets its counter), then the clusters' partial tiles
    const size_t cnt_bytes = ((size_t)tiles * plan.cs * sizeof(int) + 255) & ~(size_t)255;
    const size_t need = cnt_bytes + (size_t)tiles * plan.Q * kTcBM * 128 * sizeof(float);
    e = ws.reserve(need, s);
    if (e != cudaSuccess) return note_cuda(e);
    if (ws.ptr != g_ctx.fused_zero_ptr || cnt_bytes > g_ctx.fused_zeroed) {
      e = cudaMemsetAsync(ws.ptr, 0, cnt_bytes, s);
      if (e != cudaSuccess) return note_cuda(e);
      g_ctx.fused_zero_ptr = ws.ptr;
      g_ctx.fused_zeroed = cnt_bytes;
    }
    fp.cnt = static_cast<int *>(ws.ptr);
    fp.slots = reinterpret_cast<float *>(static_cast<uint8_t *>(ws.ptr) + cnt_bytes);
  }
  e = launch_fused(kind == kTcSplitBf16x6, fp, plan.cs, g_ctx.d_err, s);
  return note_cuda(e);
}

}  // namespace mm

extern "C" mm_status mm_tune_query_splitk(int64_t n, int64_t m, int64_t p, int *tiles,
                                          int *slices, int *clusters, int *cluster_size) {
  if (!g_ctx.inited) return MM_ENOTINIT;
  if (n < 0 || m < 0 || p < 0) return MM_EINVAL;
  FusedPlan f{0, 0, 0};
  int64_t t = 0;
  if (n > 0 && m > 0 && p > 0) {
    f = fused_plan(n, m, p, split_kind_for(m));
    t = f.S > 0 ? ceil_div(n, kTcBM) * ceil_div(p, 128) : 0;
  }
  if (tiles) *tiles = (int)t;
  if (slices) *slices = f.S;
  if (clusters) *clusters = f.Q;
  if (cluster_size) *cluster_size = f.cs;
  return MM_OK;
}
