// Plain SIMT GEMM on the CUDA cores: C = A.B with FMA in the element type.
//
// Paper anchor: Listing 4 (shared-memory tiling: every block stages a tile of
// A and a tile of B in shared memory per step along the inner dimension and
// each thread accumulates its outputs from the staged tiles).  This is that
// scheme sized for sm_103a: larger tiles, a register block of outputs per
// thread (8 x 8 in FP32, 4 x 4 in FP64), 16-byte vector loads from global
// memory, double-buffered shared memory (one barrier per K slice), and
// predicated edges so any n, m, p works (the listing needs multiples of 16).
//
// Every output is accumulated by one thread with r ascending, as in the
// definition of the Cauchy product.  Products with too few output tiles to
// fill the SMs (skinny ones above all) are cut along K into S slices (64 x 64
// tiles, or 128 x 128 for FP32 products at least 128 wide both ways): each
// slice's partial product in that order, then the S
// partials of each entry added in a fixed grouping and order by a second
// kernel.
#include <algorithm>
#include <type_traits>

#include "mm_internal.h"

namespace mm {
namespace {

template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; };
template <> struct Vec16<double> { using type = double2; };

template <typename T, int BM, int BN, int BK, int TM, int TN>
struct SimtShape {
  static constexpr int W = 16 / (int)sizeof(T);  // elements per 16-byte vector
  static constexpr int NTX = BN / TN, NTY = BM / TM;
  static constexpr int NT = NTX * NTY;
  // FP32: A's shared tile is unpadded and its 4-float groups are XOR-swizzled
  // by the K index (conflict-free transposing stores, aligned 16-byte reads);
  // FP64: rows padded by one 16-byte vector
  static constexpr bool SWZ = sizeof(T) == 4 && BK == 16 && BM % 32 == 0;
  static constexpr int APAD = SWZ ? 0 : W;
  static constexpr int VA = BM * BK / W / NT;     // vectors of A per thread and K slice
  static constexpr int VB = BK * BN / W / NT;     // vectors of B per thread and K slice
  // a thread's fragment: FA 16-byte vectors of A (rows BM / FA apart) and FB of
  // B (columns BN / FB apart) per K index
  static constexpr int FA = TM / W, FB = TN / W;
  // FP32 tiles of up to 64 outputs per thread fit two blocks per SM (at most
  // 128 registers per thread); larger ones and FP64 take one
  static constexpr int MIN_BLOCKS = (sizeof(T) == 4 && TM * TN <= 64) ? 2 : 1;
  static_assert(TM % W == 0 && TN % W == 0, "fragments of whole 16-byte vectors");
  static_assert(NT == 256, "launched with 256 threads");
  static_assert(VA >= 1 && VB >= 1 && VA * W * NT == BM * BK && VB * W * NT == BK * BN,
                "whole vectors per thread");
};

// Loads W consecutive elements of row `row`, columns col..col+W-1 of a
// row-major matrix (rows x cols, leading dimension ld), zero outside.
template <typename T, bool VEC>
__device__ __forceinline__ void load_vec(const T *__restrict__ X, int64_t ld,
                                         int64_t rows, int64_t cols,
                                         int64_t row, int64_t col, T (&v)[16 / sizeof(T)]) {
  constexpr int W = 16 / (int)sizeof(T);
  if (row < rows && col + W <= cols) {
    if (VEC) {
      typename Vec16<T>::type t = *reinterpret_cast<const typename Vec16<T>::type *>(X + row * ld + col);
      const T *tp = reinterpret_cast<const T *>(&t);
#pragma unroll
      for (int e = 0; e < W; e++) v[e] = tp[e];
    } else {
#pragma unroll
      for (int e = 0; e < W; e++) v[e] = X[row * ld + col + e];
    }
  } else {
#pragma unroll
    for (int e = 0; e < W; e++)
      v[e] = (row < rows && col + e < cols) ? X[row * ld + col + e] : T(0);
  }
}

// One BM x BN output tile.  EDGE = false: an interior tile of aligned
// operands (the tile inside C, m a multiple of BK): every load is a 16-byte
// vector through a pointer advanced by one K slice per step, no bounds checks.
// EDGE = true: predicated loads and stores for ragged edges and unaligned
// operands.
// A has leading dimension lda and K length kb (a K slice of a longer A when
// kb < lda); B has kb rows.  EPI: the stores apply the epilogue epi (C may
// then be the epilogue's D, so C is not declared unaliased).
template <typename T, bool EPI>
using OutPtr = std::conditional_t<EPI, T *, T *__restrict__>;

template <typename T, int BM, int BN, int BK, int TM, int TN, bool VEC, bool EDGE, bool EPI>
__device__ __forceinline__ void simt_tile(const T *__restrict__ A, const T *__restrict__ B,
                                          OutPtr<T, EPI> C, int64_t n, int64_t lda, int64_t kb,
                                          int64_t p,
                                          int64_t tile_m, int64_t tile_n,
                                          T (&As)[2][BK][BM + SimtShape<T, BM, BN, BK, TM, TN>::APAD],
                                          T (&Bs)[2][BK][BN], const EpiT<T> &epi) {
  using S = SimtShape<T, BM, BN, BK, TM, TN>;
  constexpr int W = S::W;
  using V = typename Vec16<T>::type;

  const int tid = threadIdx.x;
  const int tx = tid % S::NTX, ty = tid / S::NTX;
  const int64_t m0 = tile_m * BM, n0 = tile_n * BN;

  // global -> shared mapping: vector v = tid + i*NT holds A row v / (BK/W),
  // k v % (BK/W) (times W); B k v / (BN/W), columns v % (BN/W) (times W)
  constexpr int AKV = BK / W, BNV = BN / W;
  const int a_row = tid / AKV, a_kv = tid % AKV;
  const int b_k = tid / BNV, b_nv = tid % BNV;
  constexpr int ROWS_A = S::NT / AKV, KS_B = S::NT / BNV;  // strides between a thread's vectors

  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; i++)
#pragma unroll
    for (int j = 0; j < TN; j++) acc[i][j] = T(0);

  T ra[S::VA][W], rb[S::VB][W];
  const T *pa = A + (m0 + a_row) * lda + (int64_t)a_kv * W;  // interior pointers
  const T *pb = B + (int64_t)b_k * p + n0 + (int64_t)b_nv * W;
  auto load_slice = [&](int64_t k0) {
    if (!EDGE) {
#pragma unroll
      for (int i = 0; i < S::VA; i++)
        *reinterpret_cast<V *>(ra[i]) = *reinterpret_cast<const V *>(pa + (int64_t)i * ROWS_A * lda);
#pragma unroll
      for (int i = 0; i < S::VB; i++)
        *reinterpret_cast<V *>(rb[i]) = *reinterpret_cast<const V *>(pb + (int64_t)i * KS_B * p);
      pa += BK;
      pb += (int64_t)BK * p;
    } else {
#pragma unroll
      for (int i = 0; i < S::VA; i++)
        load_vec<T, VEC>(A, lda, n, kb, m0 + a_row + i * ROWS_A, k0 + (int64_t)a_kv * W, ra[i]);
#pragma unroll
      for (int i = 0; i < S::VB; i++)
        load_vec<T, VEC>(B, p, kb, p, k0 + b_k + i * KS_B, n0 + (int64_t)b_nv * W, rb[i]);
    }
  };
  // column of A's shared tile for row r at K index k: groups of 4 rows XOR
  // 2 * (k / 4) under SWZ (a warp's stores then hit 32 different banks)
  auto acol = [](int k, int r) {
    return S::SWZ ? ((((r >> 2) ^ (((k >> 2) & 3) << 1)) << 2) | (r & 3)) : r;
  };
  auto store_slice = [&](int buf) {
#pragma unroll
    for (int i = 0; i < S::VA; i++)
#pragma unroll
      for (int e = 0; e < W; e++)
        As[buf][a_kv * W + e][acol(a_kv * W + e, a_row + i * ROWS_A)] = ra[i][e];
#pragma unroll
    for (int i = 0; i < S::VB; i++)
      *reinterpret_cast<V *>(&Bs[buf][b_k + i * KS_B][b_nv * W]) = *reinterpret_cast<V *>(rb[i]);
  };

  const int64_t ktiles = (kb + BK - 1) / BK;
  if (ktiles > 0) {
    load_slice(0);
    store_slice(0);
  }
  __syncthreads();

  for (int64_t kt = 0; kt < ktiles; kt++) {
    const int cur = (int)(kt & 1);
    const bool more = kt + 1 < ktiles;
    if (more) load_slice((kt + 1) * BK);
#pragma unroll
    for (int k = 0; k < BK; k++) {
      T af[TM], bf[TN];
#pragma unroll
      for (int f = 0; f < S::FA; f++)
        *reinterpret_cast<V *>(&af[f * W]) =
            *reinterpret_cast<const V *>(&As[cur][k][acol(k, f * (BM / S::FA) + ty * W)]);
#pragma unroll
      for (int f = 0; f < S::FB; f++)
        *reinterpret_cast<V *>(&bf[f * W]) =
            *reinterpret_cast<const V *>(&Bs[cur][k][f * (BN / S::FB) + tx * W]);
#pragma unroll
      for (int i = 0; i < TM; i++)
#pragma unroll
        for (int j = 0; j < TN; j++) acc[i][j] = fma(af[i], bf[j], acc[i][j]);
    }
    if (more) store_slice(cur ^ 1);
    __syncthreads();
  }

  // store: rows hi*(BM/FA) + ty*W + i, columns hj*(BN/FB) + tx*W + j
#pragma unroll
  for (int hi = 0; hi < S::FA; hi++) {
#pragma unroll
    for (int i = 0; i < W; i++) {
      const int64_t row = m0 + hi * (BM / S::FA) + ty * W + i;
      if (EDGE && row >= n) continue;
#pragma unroll
      for (int hj = 0; hj < S::FB; hj++) {
        const int64_t col = n0 + hj * (BN / S::FB) + tx * W;
        T *dst = C + row * p + col;
        const T *src = &acc[hi * W + i][hj * W];
        if (!EDGE || (VEC && col + W <= p)) {
          V t;
          T *tp = reinterpret_cast<T *>(&t);
#pragma unroll
          for (int e = 0; e < W; e++) tp[e] = EPI ? epi_apply(epi, src[e], row * p + col + e) : src[e];
          *reinterpret_cast<V *>(dst) = t;
        } else {
#pragma unroll
          for (int e = 0; e < W; e++)
            if (col + e < p) dst[e] = EPI ? epi_apply(epi, src[e], row * p + col + e) : src[e];
        }
      }
    }
  }
}

// Interior tiles of aligned operands take the unchecked form.
template <typename T, int BM, int BN, int BK, int TM, int TN, bool VEC, bool EPI>
__device__ __forceinline__ void simt_tile_any(const T *__restrict__ A, const T *__restrict__ B,
                                              OutPtr<T, EPI> C, int64_t n, int64_t lda, int64_t kb,
                                              int64_t p, int64_t tile_m, int64_t tile_n,
                                              const EpiT<T> &epi) {
  __shared__ __align__(16) T As[2][BK][BM + SimtShape<T, BM, BN, BK, TM, TN>::APAD];
  __shared__ __align__(16) T Bs[2][BK][BN];
  const bool interior = VEC && (tile_m + 1) * BM <= n && (tile_n + 1) * BN <= p && kb % BK == 0;
  if (interior)
    simt_tile<T, BM, BN, BK, TM, TN, VEC, false, EPI>(A, B, C, n, lda, kb, p, tile_m, tile_n, As, Bs,
                                                 epi);
  else
    simt_tile<T, BM, BN, BK, TM, TN, VEC, true, EPI>(A, B, C, n, lda, kb, p, tile_m, tile_n, As, Bs,
                                                epi);
}

template <typename T, int BM, int BN, int BK, int TM, int TN, bool VEC, bool EPI>
__global__ void __launch_bounds__(256, (SimtShape<T, BM, BN, BK, TM, TN>::MIN_BLOCKS))
simt_gemm_kernel(const T *__restrict__ A, const T *__restrict__ B, OutPtr<T, EPI> C,
                 int64_t n, int64_t m, int64_t p, const int *__restrict__ run_if, EpiT<T> epi) {
  // run_if: a device word; when given, the product runs only where it is set
  if (run_if != nullptr && *reinterpret_cast<const volatile int *>(run_if) == 0) return;
  simt_tile_any<T, BM, BN, BK, TM, TN, VEC, EPI>(A, B, C, n, m, m, p, blockIdx.y, blockIdx.x, epi);
}

// K slice blockIdx.z (K values [z ks, min((z + 1) ks, m))) of a product,
// into part + z n p (C's layout).  ks is a multiple of BK, so the slice's
// first column of A keeps A's 16-byte alignment.  epi applies when the one
// slice writes C itself (S = 1), and is off otherwise.
template <typename T, int BM, int BN, int BK, int TM, int TN, bool VEC, bool EPI>
__global__ void __launch_bounds__(256, (SimtShape<T, BM, BN, BK, TM, TN>::MIN_BLOCKS))
simt_splitk_kernel(const T *__restrict__ A, const T *__restrict__ B, OutPtr<T, EPI> part,
                   int64_t n, int64_t m, int64_t p, int64_t ks, const int *__restrict__ run_if,
                   EpiT<T> epi) {
  // launched as a programmatic dependent of the previous kernel on the
  // stream: resident early, it reads nothing before that kernel has finished
  // and its writes are visible; the sum kernel may then be scheduled
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  // run_if: a device word; when given, the product runs only where it is set
  if (run_if != nullptr && *reinterpret_cast<const volatile int *>(run_if) == 0) return;
  const int64_t k0 = (int64_t)blockIdx.z * ks;
  const int64_t kb = min(ks, m - k0);
  simt_tile_any<T, BM, BN, BK, TM, TN, VEC, EPI>(A + k0, B + k0 * p, part + (int64_t)blockIdx.z * n * p,
                                            n, m, kb, p, blockIdx.y, blockIdx.x, epi);
}

// C = sum over s of part[s] for the np entries, 32 consecutive entries per
// block (the loads of a slice coalesce): warp g adds slices [g S / G,
// (g + 1) S / G) in order (G = min(8, S)), then the G partial sums are added
// in the order g = 0, 1, ..., G - 1; the epilogue epi is applied to the sum.
template <typename T>
__global__ void __launch_bounds__(256)
splitk_sum_kernel(const T *__restrict__ part, int S, int64_t np, T *C,
                  const int *__restrict__ run_if, EpiT<T> epi) {
  __shared__ T ps[8][32];
  asm volatile("griddepcontrol.wait;" ::: "memory");  // the slices' partials are written
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (run_if != nullptr && *reinterpret_cast<const volatile int *>(run_if) == 0) return;
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int G = min(8, S);
  const int64_t i = (int64_t)blockIdx.x * 32 + lane;
  if (g < G && i < np) {
    const int s0 = (int)((int64_t)g * S / G), s1 = (int)((int64_t)(g + 1) * S / G);
    T acc = part[(int64_t)s0 * np + i];
#pragma unroll 8
    for (int s = s0 + 1; s < s1; s++) acc += part[(int64_t)s * np + i];
    ps[g][lane] = acc;
  }
  __syncthreads();
  if (g == 0 && i < np) {
    T acc = ps[0][lane];
    for (int gg = 1; gg < G; gg++) acc += ps[gg][lane];
    C[i] = epi_apply(epi, acc, i);
  }
}

// Grouped form: one block per output tile over all problems of a table; the
// block finds its problem by binary search over the tile prefix.
template <typename T, int BM, int BN, int BK, int TM, int TN, bool VEC>
__global__ void __launch_bounds__(256, (SimtShape<T, BM, BN, BK, TM, TN>::MIN_BLOCKS))
simt_grouped_kernel(const SimtProb *__restrict__ probs, int nprobs) {
  const int t = blockIdx.x;
  int lo = 0, hi = nprobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (probs[mid].tile_start <= t) lo = mid; else hi = mid - 1;
  }
  const SimtProb &pr = probs[lo];
  const int local = t - pr.tile_start;
  simt_tile_any<T, BM, BN, BK, TM, TN, VEC, false>(
      static_cast<const T *>(pr.A), static_cast<const T *>(pr.B), static_cast<T *>(pr.C),
      pr.n, pr.m, pr.m, pr.p, local / pr.tiles_n, local % pr.tiles_n,
      EpiT<T>{nullptr, T(1), T(0), 0});
}

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

template <typename T, int BM, int BN, int BK, int TM, int TN>
cudaError_t launch_simt(int64_t n, int64_t m, int64_t p, const T *A, const T *B, T *C,
                        cudaStream_t s, const char *name, const int *run_if, const Epi *epi) {
  constexpr int W = 16 / (int)sizeof(T);
  const int64_t gy = ceil_div(n, BM), gx = ceil_div(p, BN);
  if (gy > 65535 || gx > 2147483647LL) return cudaErrorInvalidValue;
  dim3 grid((unsigned)gx, (unsigned)gy);
  const bool vec = aligned16(A) && aligned16(B) && aligned16(C) && m % W == 0 && p % W == 0;
  const EpiT<T> e = epi_of<T>(epi);
  TraceScope ts(name, s);
  if (e.on != 0) {
    if (vec)
      simt_gemm_kernel<T, BM, BN, BK, TM, TN, true, true><<<grid, 256, 0, s>>>(A, B, C, n, m, p, run_if, e);
    else
      simt_gemm_kernel<T, BM, BN, BK, TM, TN, false, true><<<grid, 256, 0, s>>>(A, B, C, n, m, p, run_if, e);
  } else {
    if (vec)
      simt_gemm_kernel<T, BM, BN, BK, TM, TN, true, false><<<grid, 256, 0, s>>>(A, B, C, n, m, p, run_if, e);
    else
      simt_gemm_kernel<T, BM, BN, BK, TM, TN, false, false><<<grid, 256, 0, s>>>(A, B, C, n, m, p, run_if, e);
  }
  return cudaGetLastError();
}

// Launch with programmatic stream serialization: the kernel may start while
// the stream's previous kernel finishes (it waits for it with
// griddepcontrol.wait before touching memory), which hides the gap between
// the launches of small products.
template <typename... KArgs, typename... Args>
cudaError_t launch_dependent(void (*kernel)(KArgs...), dim3 grid, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(256, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <typename T, int BM, int BN, int BK, int TM, int TN>
cudaError_t launch_splitk(int64_t n, int64_t m, int64_t p, const T *A, const T *B, T *C, T *part,
                          const SimtPlan &pl, cudaStream_t s, const char *name,
                          const int *run_if, const Epi *epi) {
  constexpr int W = 16 / (int)sizeof(T);
  const int64_t gy = ceil_div(n, BM), gx = ceil_div(p, BN);
  if (gy > 65535 || gx > 2147483647LL || pl.S < 1 || pl.S > 65535) return cudaErrorInvalidValue;
  T *out = pl.S > 1 ? part : C;
  if (pl.S > 1 && part == nullptr) return cudaErrorInvalidValue;
  dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)pl.S);
  const bool vec = aligned16(A) && aligned16(B) && aligned16(out) && m % W == 0 && p % W == 0;
  const EpiT<T> ep = epi_of<T>(epi);
  // the epilogue goes with the kernel that writes C
  const EpiT<T> slice_ep = pl.S == 1 ? ep : EpiT<T>{nullptr, T(1), T(0), 0};
  cudaError_t e;
  {
    TraceScope ts(name, s);
    if (slice_ep.on != 0)
      e = vec ? launch_dependent(simt_splitk_kernel<T, BM, BN, BK, TM, TN, true, true>, grid, s, A, B, out,
                                 n, m, p, pl.ks, run_if, slice_ep)
              : launch_dependent(simt_splitk_kernel<T, BM, BN, BK, TM, TN, false, true>, grid, s, A, B, out,
                                 n, m, p, pl.ks, run_if, slice_ep);
    else
      e = vec ? launch_dependent(simt_splitk_kernel<T, BM, BN, BK, TM, TN, true, false>, grid, s, A, B, out,
                                 n, m, p, pl.ks, run_if, slice_ep)
              : launch_dependent(simt_splitk_kernel<T, BM, BN, BK, TM, TN, false, false>, grid, s, A, B, out,
                                 n, m, p, pl.ks, run_if, slice_ep);
  }
  if (e != cudaSuccess || pl.S == 1) return e;
  TraceScope ts("simt_sum", s);
  const int64_t np = n * p;
  if (ceil_div(np, 32) > 2147483647LL) return cudaErrorInvalidValue;
  return launch_dependent(splitk_sum_kernel<T>, dim3((unsigned)ceil_div(np, 32), 1, 1), s,
                          static_cast<const T *>(part), pl.S, np, C, run_if, ep);
}

}  // namespace

SimtPlan simt_plan_for(bool f64, int64_t n, int64_t m, int64_t p, int sms) {
  SimtPlan pl{0, 0, false};
  if (n <= 0 || m <= 0 || p <= 0 || sms <= 0) return pl;
  const int64_t bm = f64 ? kSimtF64BM : kSimtF32BM, bn = f64 ? kSimtF64BN : kSimtF32BN;
  // products that fill at least half of the SMs with whole tiles keep the
  // one-pass kernel
  if (2 * ceil_div(n, bm) * ceil_div(p, bn) >= sms) return pl;
  // FP32 products at least 128 wide both ways keep the 128 x 128 tiles (8 x 8
  // outputs a thread: a quarter of the shared-memory reads per FMA of the
  // 64 x 64 tiles); narrower ones and FP64 take 64 x 64
  pl.wide = !f64 && n >= 128 && p >= 128;
  const int64_t tw = pl.wide ? 128 : 64;
  const int64_t tiles = ceil_div(n, tw) * ceil_div(p, tw);
  const int64_t bk = f64 ? kSimtF64BK : kSimtF32BK;
  const size_t es = f64 ? 8 : 4;
  // at most two CTAs per SM (one wave), slices of at least 128 K values,
  // partials of at most 256 MiB
  int64_t S = std::min(2 * (int64_t)sms / tiles, m / 128);
  S = std::min<int64_t>(S, (int64_t)((size_t(256) << 20) / ((size_t)(n * p) * es)));
  S = std::max<int64_t>(1, std::min<int64_t>(S, 1024));
  const int64_t ks = ceil_div(ceil_div(m, S), bk) * bk;
  pl.S = (int)ceil_div(m, ks);
  pl.ks = ks;
  return pl;
}

SimtPlan simt_plan(bool f64, int64_t n, int64_t m, int64_t p) {
  return simt_plan_for(f64, n, m, p, sm_count());
}

size_t simt_scratch_bytes(bool f64, int64_t n, int64_t m, int64_t p) {
  const SimtPlan pl = simt_plan(f64, n, m, p);
  return pl.S > 1 ? (size_t)pl.S * (size_t)(n * p) * (f64 ? 8 : 4) : 0;
}

cudaError_t launch_simt_splitk_f32(int64_t n, int64_t m, int64_t p, const float *A, const float *B,
                                   float *C, float *part, const SimtPlan &pl, cudaStream_t s,
                                   const Epi *epi) {
  if (pl.wide)
    return launch_splitk<float, kSimtF32BM, kSimtF32BN, kSimtF32BK, 8, 8>(n, m, p, A, B, C, part, pl, s,
                                                                         "simt_f32", nullptr, epi);
  return launch_splitk<float, 64, 64, kSimtF32BK, 4, 4>(n, m, p, A, B, C, part, pl, s, "simt_f32",
                                                        nullptr, epi);
}

cudaError_t launch_simt_splitk_f64(int64_t n, int64_t m, int64_t p, const double *A,
                                   const double *B, double *C, double *part, const SimtPlan &pl,
                                   cudaStream_t s, const int *run_if, const Epi *epi) {
  return launch_splitk<double, kSimtF64BM, kSimtF64BN, kSimtF64BK, 4, 4>(n, m, p, A, B, C, part, pl, s,
                                                                         "dgemm_f64", run_if, epi);
}

cudaError_t launch_simt_f32(int64_t n, int64_t m, int64_t p, const float *A, const float *B,
                            float *C, cudaStream_t s, const Epi *epi) {
  return launch_simt<float, kSimtF32BM, kSimtF32BN, kSimtF32BK, 8, 8>(n, m, p, A, B, C, s,
                                                                      "simt_f32", nullptr, epi);
}

cudaError_t launch_simt_f64(int64_t n, int64_t m, int64_t p, const double *A, const double *B,
                            double *C, cudaStream_t s, const int *run_if, const Epi *epi) {
  return launch_simt<double, kSimtF64BM, kSimtF64BN, kSimtF64BK, 4, 4>(n, m, p, A, B, C, s,
                                                                       "dgemm_f64", run_if, epi);
}

cudaError_t launch_simt_grouped(bool f64, const SimtProb *d_probs, int nprobs, int total_tiles,
                                bool all_vec, cudaStream_t s) {
  if (total_tiles <= 0) return cudaSuccess;
  if (f64) {
    TraceScope ts("dgemm_f64", s);
    if (all_vec)
      simt_grouped_kernel<double, kSimtF64BM, kSimtF64BN, kSimtF64BK, 4, 4, true>
          <<<total_tiles, 256, 0, s>>>(d_probs, nprobs);
    else
      simt_grouped_kernel<double, kSimtF64BM, kSimtF64BN, kSimtF64BK, 4, 4, false>
          <<<total_tiles, 256, 0, s>>>(d_probs, nprobs);
  } else {
    TraceScope ts("simt_f32", s);
    if (all_vec)
      simt_grouped_kernel<float, kSimtF32BM, kSimtF32BN, kSimtF32BK, 8, 8, true>
          <<<total_tiles, 256, 0, s>>>(d_probs, nprobs);
    else
      simt_grouped_kernel<float, kSimtF32BM, kSimtF32BN, kSimtF32BK, 8, 8, false>
          <<<total_tiles, 256, 0, s>>>(d_probs, nprobs);
  }
  return cudaGetLastError();
}

}  // namespace mm

extern "C" mm_status mm_simt_plan(int64_t n, int64_t m, int64_t p, mm_dtype dt, int sms,
                                  int *slices, int64_t *slice_k, int *tile) {
  using namespace mm;
  if (n < 0 || m < 0 || p < 0 || (dt != MM_F32 && dt != MM_F64) || !slices || !slice_k || !tile)
    return MM_EINVAL;
  const bool f64 = dt == MM_F64;
  const SimtPlan pl = simt_plan_for(f64, n, m, p, sms > 0 ? sms : sm_count());
  *slices = pl.S;
  *slice_k = pl.S > 0 ? pl.ks : 0;
  *tile = pl.S > 0 ? (pl.wide ? 128 : 64) : (f64 ? kSimtF64BM : kSimtF32BM);
  return MM_OK;
}
