/*
 * CPU oracle for the dense Cauchy matrix product C = A.B.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or calls
 * this file: only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
 * leg use it.  It shares no code, header or constant with the CUDA path.
 *
 * What it computes (paper, Section "Implementacje algorytmow"):
 *   definition of the Cauchy product:  c_ij = sum_{r=1..m} a_ir * b_rj,
 *   1 <= i <= n, 1 <= j <= p  (the equation right after the section heading);
 *   sequential algorithm (Listing 1): rows i ascending, then columns j, then
 *   the inner index ascending, C(i,j) set to zero first and accumulated in place.
 * Row-major storage with leading dimension = number of columns (Listing 1:
 * A[i*m + k], B[k*p + j], C[i*p + j]).
 *
 * Readings of the paper that this file takes:
 *   - Listing 1 is garbled (broken identifiers); it is read as
 *     C[i*p + j] = sum_{k=0}^{m-1} A[i*m + k] * B[k*p + j], k ascending.
 *   - the FP64 oracle reads B through a transposed copy so the inner loop is
 *     contiguous; that moves data only, the summation order per entry is
 *     Listing 1's.
 *   - rows are split over threads in contiguous blocks; every entry is still
 *     computed by one thread in Listing 1's order, so the result does not
 *     depend on the thread count.
 * Build with -ffp-contract=off: every step is RN(RN(a*b) + s).
 *
 * Accurate checks:
 *   oracle_entries_dot2  compensated dot product "Dot2" (T. Ogita, S. M. Rump,
 *                        S. Oishi, "Accurate sum and dot product", SIAM J. Sci.
 *                        Comput. 26(6), 2005): TwoProduct by fma, TwoSum by
 *                        Knuth's branch-free formula.
 *   oracle_entries_ld    long double accumulation (64-bit significand on x86,
 *                        113-bit on aarch64).
 *   oracle_gemm_pow2_exact  exact fixed-point sum for inputs that are 0 or
 *                        +-2^k (the power-of-two stress case).
 *
 * Compile-time mutants (ORACLE_MUTANT=1..9) plant plausible mistakes; the
 * pin tests build them to show that every such mistake is caught.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>
#include <float.h>

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

int oracle_mutant(void) { return ORACLE_MUTANT; }
int oracle_ldbl_mant_dig(void) { return LDBL_MANT_DIG; }

int oracle_default_threads(void) {
  long c = sysconf(_SC_NPROCESSORS_ONLN);
  return c > 0 ? (int)c : 1;
}

/* ---------------------------------------------------------------- FP64 GEMM */

typedef struct {
  int64_t n, m, p, i0, i1;
  const double *A, *Bt;
  double *C, *absC;
} gemm_job;

static void *gemm_rows(void *arg) {
  const gemm_job *g = (const gemm_job *)arg;
  const int64_t m = g->m, p = g->p;
  for (int64_t i = g->i0; i < g->i1; i++) {
    const double *a_row = g->A + i * m;
#if ORACLE_MUTANT == 5
    double s = 0.0; /* mutant: accumulator reset once per row, not per entry */
#endif
    for (int64_t j = 0; j < p; j++) {
      const double *b_col = g->Bt + j * m;
#if ORACLE_MUTANT != 5
      double s = 0.0;
#endif
      double sa = 0.0;
#if ORACLE_MUTANT == 1
      const int64_t m_used = m > 0 ? m - 1 : 0; /* mutant: last term dropped */
#else
      const int64_t m_used = m;
#endif
      for (int64_t k = 0; k < m_used; k++) {
#if ORACLE_MUTANT == 2
        const double a = a_row[m - 1 - k]; /* mutant: A's inner index reversed */
#else
        const double a = a_row[k];
#endif
        const double b = b_col[k];
#if ORACLE_MUTANT == 3
        if (k == 0) s -= a * b; else s += a * b; /* mutant: sign of first term */
#else
        s += a * b;
#endif
#if ORACLE_MUTANT == 7
        sa += a * b; /* mutant: normaliser without absolute values */
#else
        sa += fabs(a) * fabs(b);
#endif
      }
      g->C[i * p + j] = s;
      if (g->absC) g->absC[i * p + j] = sa;
    }
  }
  return NULL;
}

/* C = A.B in FP64 (Listing 1 order); absC = |A|.|B| if absC != NULL.
 * A: n x m, B: m x p, C/absC: n x p, all row-major and dense.
 * threads <= 0 selects all online cores.  Returns 0, or -1 on allocation
 * failure. */
int oracle_gemm_f64(int64_t n, int64_t m, int64_t p, const double *A,
                    const double *B, double *C, double *absC, int threads) {
  if (n <= 0 || p <= 0) return 0;
  double *Bt = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m * p : 1));
  if (!Bt) return -1;
  for (int64_t k = 0; k < m; k++)
    for (int64_t j = 0; j < p; j++) {
#if ORACLE_MUTANT == 4
      Bt[j * m + k] = B[j * m + k]; /* mutant: B read as if stored transposed */
#else
      Bt[j * m + k] = B[k * p + j];
#endif
    }
  if (threads <= 0) threads = oracle_default_threads();
  if (threads > n) threads = (int)n;
  pthread_t *tid = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)threads);
  gemm_job *jobs = (gemm_job *)malloc(sizeof(gemm_job) * (size_t)threads);
  if (!tid || !jobs) { free(Bt); free(tid); free(jobs); return -1; }
  for (int t = 0; t < threads; t++) {
    jobs[t].n = n; jobs[t].m = m; jobs[t].p = p;
    jobs[t].i0 = n * t / threads;
    jobs[t].i1 = n * (t + 1) / threads;
    jobs[t].A = A; jobs[t].Bt = Bt; jobs[t].C = C; jobs[t].absC = absC;
  }
  char *live = (char *)calloc((size_t)threads, 1);
  for (int t = 1; t < threads; t++) {
    if (live && pthread_create(&tid[t], NULL, gemm_rows, &jobs[t]) == 0) live[t] = 1;
    else gemm_rows(&jobs[t]); /* could not start a thread: run the block here */
  }
  gemm_rows(&jobs[0]);
  for (int t = 1; t < threads; t++)
    if (live && live[t]) pthread_join(tid[t], NULL);
  free(live); free(Bt); free(tid); free(jobs);
  return 0;
}

/* --------------------------------------------------------- compensated Dot2 */

static inline void two_sum(double a, double b, double *s, double *e) {
  double x = a + b;
  double z = x - a;
  *e = (a - (x - z)) + (b - z);
  *s = x;
}

static inline void two_prod(double a, double b, double *h, double *r) {
  double x = a * b;
  *r = fma(a, b, -x);
  *h = x;
}

/* Dot2 of x (stride sx) and y (stride sy), length len: returns hi, lo with
 * hi + lo ~= the dot product to about twice the working precision. */
static void dot2(int64_t len, const double *x, int64_t sx, const double *y,
                 int64_t sy, double *hi, double *lo) {
  double p = 0.0, s = 0.0;
  for (int64_t k = 0; k < len; k++) {
    double h, r, q;
    two_prod(x[k * sx], y[k * sy], &h, &r);
    two_sum(p, h, &p, &q);
#if ORACLE_MUTANT == 8
    (void)q; (void)r; /* mutant: compensation terms dropped */
#else
    s += q + r;
#endif
  }
  double res = p + s;
  *hi = res;
  *lo = (p - res) + s;
}

/* Sampled entries c_ij (Dot2) and (|A||B|)_ij for (I[t], J[t]), t < count. */
void oracle_entries_dot2(int64_t n, int64_t m, int64_t p, const double *A,
                         const double *B, int64_t count, const int64_t *I,
                         const int64_t *J, double *hi, double *lo,
                         double *absv) {
  (void)n;
  for (int64_t t = 0; t < count; t++) {
    const double *a = A + I[t] * m;
    const double *b = B + J[t];
    dot2(m, a, 1, b, p, &hi[t], &lo[t]);
    double sa = 0.0;
    for (int64_t k = 0; k < m; k++) sa += fabs(a[k]) * fabs(b[k * p]);
    absv[t] = sa;
  }
}

/* Same entries accumulated in long double; hi = (double)sum,
 * lo = (double)(sum - hi). */
void oracle_entries_ld(int64_t n, int64_t m, int64_t p, const double *A,
                       const double *B, int64_t count, const int64_t *I,
                       const int64_t *J, double *hi, double *lo) {
  (void)n;
  for (int64_t t = 0; t < count; t++) {
    const double *a = A + I[t] * m;
    const double *b = B + J[t];
    long double s = 0.0L;
    for (int64_t k = 0; k < m; k++) s += (long double)a[k] * (long double)b[k * p];
    double h = (double)s;
    hi[t] = h;
    lo[t] = (double)(s - (long double)h);
  }
}

/* y = X.v with Dot2 per row (y = hi part), yabs = |X|.|v|.
 * X: rows x cols row-major. */
void oracle_gemv_dot2(int64_t rows, int64_t cols, const double *X,
                      const double *v, double *y, double *yabs) {
  for (int64_t i = 0; i < rows; i++) {
    double h, l;
    dot2(cols, X + i * cols, 1, v, 1, &h, &l);
    y[i] = h;
    if (yabs) {
      double sa = 0.0;
      for (int64_t k = 0; k < cols; k++) sa += fabs(X[i * cols + k]) * fabs(v[k]);
      yabs[i] = sa;
    }
  }
}

/* ------------------------------------------------------- complex product */

/* Complex C = A.B (the definition with complex entries; Table 2's "complex
 * float" column computes this product): interleaved (re, im) row-major
 * arrays of doubles, A n x m, B m x p, C n x p, Listing 1's order per entry.
 * absC (optional, real n x p) = sum_r |a_ir| |b_rj| with complex moduli. */
void oracle_cgemm_f64(int64_t n, int64_t m, int64_t p, const double *A, const double *B,
                      double *C, double *absC) {
  for (int64_t i = 0; i < n; i++)
    for (int64_t j = 0; j < p; j++) {
      double sr = 0.0, si = 0.0, sa = 0.0;
      for (int64_t k = 0; k < m; k++) {
        const double ar = A[2 * (i * m + k)], ai = A[2 * (i * m + k) + 1];
        const double br = B[2 * (k * p + j)], bi = B[2 * (k * p + j) + 1];
        sr += ar * br - ai * bi;
#if ORACLE_MUTANT == 9
        si += ar * bi - ai * br; /* mutant: sign of a cross term */
#else
        si += ar * bi + ai * br;
#endif
        sa += sqrt(ar * ar + ai * ai) * sqrt(br * br + bi * bi);
      }
      C[2 * (i * p + j)] = sr;
      C[2 * (i * p + j) + 1] = si;
      if (absC) absC[i * p + j] = sa;
    }
}

/* ------------------------------------------------------ exact power-of-two */

/* Exact C = A.B for entries that are 0 or +-2^k.  Every product 2^(ka+kb)
 * must satisfy ka+kb >= -shift and ka+kb+shift <= 100, and m <= 2^20, so the
 * fixed-point sum (unit 2^-shift) fits in a signed 128-bit integer.  Output:
 * hi = the exact value rounded to double, lo = rounded remainder.
 * Returns 0, or the 1-based flat index of the first offending input entry as
 * a negative number. */
int64_t oracle_gemm_pow2_exact(int64_t n, int64_t m, int64_t p,
                               const double *A, const double *B, int shift,
                               double *hi, double *lo) {
  if (m > (1 << 20)) return -1;
  for (int64_t i = 0; i < n; i++) {
    for (int64_t j = 0; j < p; j++) {
      __int128 acc = 0;
      for (int64_t k = 0; k < m; k++) {
        double a = A[i * m + k], b = B[k * p + j];
        if (a == 0.0 || b == 0.0) continue;
        int ea, eb;
        double fa = frexp(a, &ea), fb = frexp(b, &eb);
        if (fabs(fa) != 0.5) return -(i * m + k + 1);
        if (fabs(fb) != 0.5) return -(n * m + k * p + j + 1);
        int e = (ea - 1) + (eb - 1) + shift; /* a*b = +-2^(ea-1+eb-1) */
        if (e < 0 || e > 100) return -(i * m + k + 1);
        __int128 term = (__int128)1 << e;
        if ((fa < 0) != (fb < 0)) acc -= term; else acc += term;
      }
      /* split acc into two doubles exactly: acc = h*2^64 + l (l unsigned) */
      int neg = acc < 0;
      unsigned __int128 u = neg ? (unsigned __int128)(-acc) : (unsigned __int128)acc;
      /* correctly rounded conversion by gcc, then remainder */
      double h = (double)u;
      unsigned __int128 hu = (unsigned __int128)h;
      double r;
      if (hu >= u) r = -(double)(hu - u); else r = (double)(u - hu);
      h = ldexp(h, -shift);
      r = ldexp(r, -shift);
      hi[i * p + j] = neg ? -h : h;
      lo[i * p + j] = neg ? -r : r;
    }
  }
  return 0;
}
