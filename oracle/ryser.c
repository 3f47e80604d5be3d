/*
 * Plain CPU oracle for matrix permanents.
 *
 * TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the
 * CPU-baseline leg of the benchmark are the only code that may load this
 * library.  The library path (the CUDA kernels behind include/perm.h) never
 * calls it, and the two share no source.
 *
 * Every routine is a slow, direct transcription of a passage of
 * arXiv:2502.16577 ("SUperman: Efficient Permanent Computation on GPUs"):
 *
 *   oracle_gray, oracle_changed_bit    Sec. 2, Table 1: Gray_g = g xor (g >> 1),
 *                                      changed bit = log2(Gray_g xor Gray_{g-1}).
 *   oracle_cbl                         Sec. 3.1.1: CBL_k = CBL_{k-1} + [k-1] + CBL_{k-1}^R.
 *   oracle_ryser_f64_range             Alg. 1 (RYSER with the Nijenhuis-Wilf row
 *                                      vector x, Eq. nwx) over a sub-range of g, split
 *                                      over threads as in Alg. 3 (PARRYSER); thread
 *                                      partials and the outer sum in double-double
 *                                      ("quad as two doubles", Sec. 5).
 *   oracle_ryser_dd_range              Alg. 1 with x and prod also in double-double:
 *                                      the high-precision reference of Sec. 5's
 *                                      accuracy study.
 *   oracle_ryser_c128_range            Alg. 1 over complex entries (complex support is
 *                                      claimed in Secs. 1 and 7; same recurrence in C).
 *   oracle_ryser_dd_stats_range,       Alg. 1 in double-double (real; complex with the
 *   oracle_ryser_cdd_range             four-multiply product), also returning the
 *                                      magnitude sums that scale the rounding errors
 *                                      studied in Sec. 5 (sum of |terms|, and the same
 *                                      with one factor replaced by its row's size).
 *   oracle_spa_ryser_f64_range         Alg. 2 (SPARYSER): CRS for the row sums, CCS for
 *                                      the column updates.
 *   oracle_ryser_bin_plain             Eq. 2 (Ryser over all 2^n column subsets, no
 *                                      halving) in wrap-around 128-bit integers.
 *   oracle_ryser_bin_range             Alg. 1 over the doubled rows x' = 2x, exact,
 *                                      wrap-around 128-bit integers.
 *   oracle_perm_dp_*                   Eq. 1 expanded row by row over column subsets
 *                                      (independent of Ryser and of Gray codes).
 *
 * Readings of the paper taken here (where its text is silent or garbled):
 *   - Columns are 0-based; the paper's column n is column n-1 here and is in
 *     every subset; Gray bit j selects column j (Sec. 2, "counting starts from
 *     the least significant bit").
 *   - The g = 0 term (Alg. 1's product of the start state) belongs to the first range;
 *     Alg. 3 omits it.  Ranges are half-open: [g_begin, g_end) within
 *     [0, 2^(n-1)); Alg. 3's inclusive end is read as exclusive.
 *   - Alg. 2's loop body "row <- rids[ptr]; val <- cvals[ptr]" is completed
 *     with "x[row] <- x[row] + s * val".
 *   - perm of the 0x0 matrix is 1 (empty product).
 *
 * Parity is pinned by tests/test_oracle_*.py against Table 1, the CBL
 * recursion, brute force over permutations (Eq. 1), closed forms and
 * invariants; no routine here is "parity unpinned".
 *
 * Build: plain C11 + pthreads, -ffp-contract=off (no fused multiply-add
 * except the explicit fma() of the double-double product).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_NMAX 64

/* ORACLE_MUTANT selects one planted mistake (tests/test_oracle_mutants.py
 * checks that the pins catch each); 0, the default, is the oracle itself. */
#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

/* ---------------------------------------------------------------- Gray code */

uint64_t oracle_gray(uint64_t g) { return g ^ (g >> 1); }

/* log2(Gray_g xor Gray_{g-1}) for g >= 1 (Table 1, "Changed Bits" column). */
int oracle_changed_bit(uint64_t g) {
  uint64_t d = oracle_gray(g) ^ oracle_gray(g - 1);
  int j = 0;
  while (d > 1) {
    d >>= 1;
    ++j;
  }
  return j;
}

/* CBL_k by the reflection recursion of Sec. 3.1.1; out has room for 2^k - 1. */
int oracle_cbl(int k, int* out) {
  if (k < 1 || k > 24) return -1;
  int len = 1;
  out[0] = 0; /* CBL_1 = [0] */
  for (int b = 2; b <= k; ++b) {
    out[len] = b - 1;
    for (int t = 0; t < len; ++t) out[len + 1 + t] = out[len - 1 - t];
    len = 2 * len + 1;
  }
  return len;
}

/* ------------------------------------------------------------ double-double */

typedef struct {
  double hi, lo;
} dd_t;

static void two_sum(double a, double b, double* s, double* e) {
  double x = a + b;
  double bv = x - a;
  double av = x - bv;
  *e = (a - av) + (b - bv);
  *s = x;
}

static dd_t dd_from_sum(double s, double e) {
  dd_t r;
  double h = s + e;
  r.lo = e - (h - s);
  r.hi = h;
  return r;
}

static dd_t dd_add(dd_t a, dd_t b) {
  double s, e;
  two_sum(a.hi, b.hi, &s, &e);
  e += a.lo + b.lo;
  return dd_from_sum(s, e);
}

static dd_t dd_add_d(dd_t a, double b) {
  double s, e;
  two_sum(a.hi, b, &s, &e);
  e += a.lo;
  return dd_from_sum(s, e);
}

static dd_t dd_neg(dd_t a) {
  dd_t r = {-a.hi, -a.lo};
  return r;
}

static dd_t dd_mul(dd_t a, dd_t b) {
  double p = a.hi * b.hi;
  double e = fma(a.hi, b.hi, -p);
  e += a.hi * b.lo + a.lo * b.hi;
  return dd_from_sum(p, e);
}

static const dd_t DD_ZERO = {0.0, 0.0};

/* -------------------------------------------------------- thread scaffolding */

typedef struct {
  const void* ctx;
  uint64_t start, end; /* half-open sub-range of g */
  void (*body)(const void* ctx, uint64_t start, uint64_t end, void* out);
  void* out;
} job_t;

static void* job_main(void* p) {
  job_t* j = (job_t*)p;
  if (j->start < j->end) j->body(j->ctx, j->start, j->end, j->out);
  return NULL;
}

/* Alg. 3: chnksz = ceil(range / tau); thread tid gets [start, end). */
static int run_chunks(const void* ctx, uint64_t g0, uint64_t g1, int tau,
                      void (*body)(const void*, uint64_t, uint64_t, void*), void* outs, size_t out_size) {
  if (tau < 1) tau = 1;
  if (tau > 1024) tau = 1024;
  uint64_t range = g1 - g0;
  uint64_t chnksz = (range + (uint64_t)tau - 1) / (uint64_t)tau;
  if (chnksz == 0) chnksz = 1;
  job_t* jobs = (job_t*)calloc((size_t)tau, sizeof(job_t));
  pthread_t* th = (pthread_t*)calloc((size_t)tau, sizeof(pthread_t));
  if (!jobs || !th) {
    free(jobs);
    free(th);
    return -1;
  }
  for (int t = 0; t < tau; ++t) {
    uint64_t s = g0 + chnksz * (uint64_t)t;
    uint64_t e = s + chnksz;
    if (s > g1) s = g1;
    if (e > g1) e = g1;
    jobs[t].ctx = ctx;
    jobs[t].start = s;
    jobs[t].end = e;
    jobs[t].body = body;
    jobs[t].out = (char*)outs + out_size * (size_t)t;
  }
  int nstarted = 0;
  for (int t = 1; t < tau; ++t) {
    if (pthread_create(&th[t], NULL, job_main, &jobs[t]) != 0) break;
    ++nstarted;
  }
  job_main(&jobs[0]);
  for (int t = 1; t <= nstarted; ++t) pthread_join(th[t], NULL);
  for (int t = nstarted + 1; t < tau; ++t) job_main(&jobs[t]); /* thread creation failed: run inline */
  free(jobs);
  free(th);
  return 0;
}

/* ------------------------------------------------- Alg. 1 / Alg. 3, real FP64 */

typedef struct {
  const double* A; /* row-major n x n: a_{i,j} = A[i*n + j] */
  int n;
} real_ctx_t;

/* Alg. 1, start state: x[i] = a_{i,n} - (sum_j a_{i,j}) / 2 (paper's column n). */
static void nw_start_f64(const double* A, int n, double* x) {
  for (int i = 0; i < n; ++i) {
    double sum = 0.0;
    for (int j = 0; j < n; ++j) sum += A[i * n + j];
#if ORACLE_MUTANT == 2
    x[i] = A[i * n + 0] - sum / 2.0; /* planted: wrong column index */
#elif ORACLE_MUTANT == 3
    x[i] = A[i * n + (n - 1)] - sum; /* planted: dropped halving */
#else
    x[i] = A[i * n + (n - 1)] - sum / 2.0;
#endif
  }
}

/* Alg. 3, per-thread start: add every column whose bit is set in Gray_{start-1}. */
static void gray_state_f64(const double* A, int n, uint64_t g, double* x) {
  uint64_t G = oracle_gray(g);
  for (int j = 0; j < n - 1; ++j)
    if ((G >> j) & 1u)
      for (int i = 0; i < n; ++i) x[i] += A[i * n + j];
}

static void ryser_f64_body(const void* vctx, uint64_t s, uint64_t e, void* out) {
  const real_ctx_t* c = (const real_ctx_t*)vctx;
  const double* A = c->A;
  int n = c->n;
  double x[ORACLE_NMAX];
  dd_t p = DD_ZERO;
  nw_start_f64(A, n, x);
  uint64_t start = s;
  if (s == 0) { /* Alg. 1: p <- prod_i x[i] for the empty subset (g = 0) */
    double prod = 1.0;
    for (int i = 0; i < n; ++i) prod *= x[i];
#if ORACLE_MUTANT != 7
    p = dd_add_d(p, prod);
#endif
    start = 1;
  }
#if ORACLE_MUTANT == 6
  if (start < e) gray_state_f64(A, n, start, x); /* planted: off-by-one start state */
#else
  if (start < e) gray_state_f64(A, n, start - 1, x);
#endif
  for (uint64_t g = start; g < e; ++g) {
    int j = oracle_changed_bit(g);                           /* Alg. 1: changed column */
#if ORACLE_MUTANT == 5
    double sg = 1.0 - 2.0 * (double)((oracle_gray(g) >> j) & 1u); /* planted: sign flipped */
#else
    double sg = 2.0 * (double)((oracle_gray(g) >> j) & 1u) - 1.0; /* +1 enters, -1 leaves */
#endif
    double prod = 1.0;
    for (int i = 0; i < n; ++i) {                            /* update x, multiply */
      x[i] = x[i] + sg * A[i * n + j];
      prod = prod * x[i];
    }
#if ORACLE_MUTANT == 1
    p = dd_add_d(p, prod); /* planted: (-1)^g dropped */
#else
    p = (g & 1u) ? dd_add_d(p, -prod) : dd_add_d(p, prod); /* p += (-1)^g prod */
#endif
  }
  *(dd_t*)out = p;
}

static int check_range(int n, uint64_t g0, uint64_t g1) {
  if (n < 1 || n > ORACLE_NMAX - 1) return -1;
  uint64_t N = 1ull << (n - 1);
  if (g0 > g1 || g1 > N) return -2;
  return 0;
}

/*
 * Sum over g in [g0, g1) of (-1)^g prod_i x_i(g), where x_i(g) is Alg. 1's
 * row vector after the subsets up to Gray_g (x_i(0) = a_{i,n} - r_i/2).
 * perm(A) = 2 (-1)^(n-1) times the sum over [0, 2^(n-1)).  Result in
 * double-double (out[0] = hi, out[1] = lo).
 */
int oracle_ryser_f64_range(const double* A, int n, uint64_t g0, uint64_t g1, int threads, double* out) {
  int rc = check_range(n, g0, g1);
  if (rc) return rc;
  real_ctx_t ctx = {A, n};
  int tau = threads < 1 ? 1 : threads;
  dd_t* parts = (dd_t*)calloc((size_t)tau, sizeof(dd_t));
  if (!parts) return -3;
  if (run_chunks(&ctx, g0, g1, tau, ryser_f64_body, parts, sizeof(dd_t))) {
    free(parts);
    return -3;
  }
  dd_t tot = DD_ZERO;
  for (int t = 0; t < tau; ++t) tot = dd_add(tot, parts[t]); /* outer sum, fixed order */
  free(parts);
  out[0] = tot.hi;
  out[1] = tot.lo;
  return 0;
}

/* Alg. 1, result: p * (4 (n mod 2) - 2).  n = 0 gives 1. */
int oracle_perm_f64(const double* A, int n, int threads, double* out) {
  if (n == 0) {
    out[0] = 1.0;
    return 0;
  }
  double s[2];
  int rc = oracle_ryser_f64_range(A, n, 0, 1ull << (n - 1), threads, s);
  if (rc) return rc;
#if ORACLE_MUTANT == 4
  double f = 2.0; /* planted: (-1)^(n-1) dropped from the final factor */
#else
  double f = 4.0 * (double)(n % 2) - 2.0;
#endif
  out[0] = (s[0] + s[1]) * f;
  return 0;
}

/* ------------------------------------------- Alg. 1, x and prod double-double */

static void ryser_dd_body(const void* vctx, uint64_t s, uint64_t e, void* out) {
  const real_ctx_t* c = (const real_ctx_t*)vctx;
  const double* A = c->A;
  int n = c->n;
  dd_t x[ORACLE_NMAX];
  for (int i = 0; i < n; ++i) {
    dd_t sum = DD_ZERO;
    for (int j = 0; j < n; ++j) sum = dd_add_d(sum, A[i * n + j]);
    dd_t half = {sum.hi / 2.0, sum.lo / 2.0}; /* exact: scaling by 1/2 */
    x[i] = dd_add_d(dd_neg(half), A[i * n + (n - 1)]);
  }
  dd_t p = DD_ZERO;
  uint64_t start = s;
  if (s == 0) {
    dd_t prod = {1.0, 0.0};
    for (int i = 0; i < n; ++i) prod = dd_mul(prod, x[i]);
    p = dd_add(p, prod);
    start = 1;
  }
  if (start < e) {
    uint64_t G = oracle_gray(start - 1);
    for (int j = 0; j < n - 1; ++j)
      if ((G >> j) & 1u)
        for (int i = 0; i < n; ++i) x[i] = dd_add_d(x[i], A[i * n + j]);
  }
  for (uint64_t g = start; g < e; ++g) {
    int j = oracle_changed_bit(g);
    double sg = 2.0 * (double)((oracle_gray(g) >> j) & 1u) - 1.0;
    dd_t prod = {1.0, 0.0};
    for (int i = 0; i < n; ++i) {
      x[i] = dd_add_d(x[i], sg * A[i * n + j]);
      prod = dd_mul(prod, x[i]);
    }
    p = (g & 1u) ? dd_add(p, dd_neg(prod)) : dd_add(p, prod);
  }
  *(dd_t*)out = p;
}

int oracle_ryser_dd_range(const double* A, int n, uint64_t g0, uint64_t g1, int threads, double* out) {
  int rc = check_range(n, g0, g1);
  if (rc) return rc;
  real_ctx_t ctx = {A, n};
  int tau = threads < 1 ? 1 : threads;
  dd_t* parts = (dd_t*)calloc((size_t)tau, sizeof(dd_t));
  if (!parts) return -3;
  if (run_chunks(&ctx, g0, g1, tau, ryser_dd_body, parts, sizeof(dd_t))) {
    free(parts);
    return -3;
  }
  dd_t tot = DD_ZERO;
  for (int t = 0; t < tau; ++t) tot = dd_add(tot, parts[t]);
  free(parts);
  out[0] = tot.hi;
  out[1] = tot.lo;
  return 0;
}

/* perm in double-double: out[0] + out[1]. */
int oracle_perm_dd(const double* A, int n, int threads, double* out) {
  if (n == 0) {
    out[0] = 1.0;
    out[1] = 0.0;
    return 0;
  }
  double s[2];
  int rc = oracle_ryser_dd_range(A, n, 0, 1ull << (n - 1), threads, s);
  if (rc) return rc;
  double f = 4.0 * (double)(n % 2) - 2.0; /* exact power-of-two scaling */
  out[0] = s[0] * f;
  out[1] = s[1] * f;
  return 0;
}

/* ------------------------------------------------------- Alg. 1, complex128 */

typedef struct {
  const double* A; /* row-major n x n of (re, im) pairs */
  int n;
} cplx_ctx_t;

typedef struct {
  dd_t re, im;
} cdd_t;

static void ryser_c128_body(const void* vctx, uint64_t s, uint64_t e, void* out) {
  const cplx_ctx_t* c = (const cplx_ctx_t*)vctx;
  const double* A = c->A;
  int n = c->n;
  double xr[ORACLE_NMAX], xi[ORACLE_NMAX];
  for (int i = 0; i < n; ++i) {
    double sr = 0.0, si = 0.0;
    for (int j = 0; j < n; ++j) {
      sr += A[2 * (i * n + j)];
      si += A[2 * (i * n + j) + 1];
    }
    xr[i] = A[2 * (i * n + n - 1)] - sr / 2.0;
    xi[i] = A[2 * (i * n + n - 1) + 1] - si / 2.0;
  }
  cdd_t p = {DD_ZERO, DD_ZERO};
  uint64_t start = s;
  if (s == 0) {
    double pr = 1.0, pi = 0.0;
    for (int i = 0; i < n; ++i) {
      double tr = pr * xr[i] - pi * xi[i];
      double ti = pr * xi[i] + pi * xr[i];
      pr = tr;
      pi = ti;
    }
    p.re = dd_add_d(p.re, pr);
    p.im = dd_add_d(p.im, pi);
    start = 1;
  }
  if (start < e) {
    uint64_t G = oracle_gray(start - 1);
    for (int j = 0; j < n - 1; ++j)
      if ((G >> j) & 1u)
        for (int i = 0; i < n; ++i) {
          xr[i] += A[2 * (i * n + j)];
          xi[i] += A[2 * (i * n + j) + 1];
        }
  }
  for (uint64_t g = start; g < e; ++g) {
    int j = oracle_changed_bit(g);
    double sg = 2.0 * (double)((oracle_gray(g) >> j) & 1u) - 1.0;
    double pr = 1.0, pi = 0.0;
    for (int i = 0; i < n; ++i) {
      xr[i] = xr[i] + sg * A[2 * (i * n + j)];
      xi[i] = xi[i] + sg * A[2 * (i * n + j) + 1];
      double tr = pr * xr[i] - pi * xi[i];
      double ti = pr * xi[i] + pi * xr[i];
      pr = tr;
      pi = ti;
    }
    if (g & 1u) {
      pr = -pr;
      pi = -pi;
    }
    p.re = dd_add_d(p.re, pr);
    p.im = dd_add_d(p.im, pi);
  }
  *(cdd_t*)out = p;
}

/* out = {re.hi, re.lo, im.hi, im.lo} of the unscaled range sum. */
int oracle_ryser_c128_range(const double* A, int n, uint64_t g0, uint64_t g1, int threads, double* out) {
  int rc = check_range(n, g0, g1);
  if (rc) return rc;
  cplx_ctx_t ctx = {A, n};
  int tau = threads < 1 ? 1 : threads;
  cdd_t* parts = (cdd_t*)calloc((size_t)tau, sizeof(cdd_t));
  if (!parts) return -3;
  if (run_chunks(&ctx, g0, g1, tau, ryser_c128_body, parts, sizeof(cdd_t))) {
    free(parts);
    return -3;
  }
  dd_t re = DD_ZERO, im = DD_ZERO;
  for (int t = 0; t < tau; ++t) {
    re = dd_add(re, parts[t].re);
    im = dd_add(im, parts[t].im);
  }
  free(parts);
  out[0] = re.hi;
  out[1] = re.lo;
  out[2] = im.hi;
  out[3] = im.lo;
  return 0;
}

int oracle_perm_c128(const double* A, int n, int threads, double* out) {
  if (n == 0) {
    out[0] = 1.0;
    out[1] = 0.0;
    return 0;
  }
  double s[4];
  int rc = oracle_ryser_c128_range(A, n, 0, 1ull << (n - 1), threads, s);
  if (rc) return rc;
  double f = 4.0 * (double)(n % 2) - 2.0;
  out[0] = (s[0] + s[1]) * f;
  out[1] = (s[2] + s[3]) * f;
  return 0;
}

/* ------------------------ Alg. 1 in double-double, with rounding statistics */
/*
 * Sec. 5 relates the accuracy of the sweep to the size of its terms.  The two
 * sweeps below run Alg. 1 with x and every product in double-double (real, and
 * complex with the standard four-multiply product) and also return two sums
 * of magnitudes that scale rounding errors:
 *   S = sum_g |prod_i x_i(g)|                        (the size of every term)
 *   W = sum_g sum_i R_i prod_{k != i} |x_k(g)|,  R_i = sum_j |a_ij|
 * A relative error eps in every term moves the range sum by at most eps S; an
 * error of at most eps R_i in each x_i(g) moves it by at most about eps W
 * (first order).  |.| is the modulus for complex entries.  Both sums are
 * formed in binary64 per step from the leading words and added up in
 * double-double: they are magnitudes for error bounds, not exact values.
 */

typedef struct {
  dd_t p, s, w;
} dd_stats_t;

/* S and W of one term from the moduli xa[i] = |x_i(g)| and R[i]. */
static void stats_step(const double* xa, const double* R, int n, dd_stats_t* st) {
  double pre[ORACLE_NMAX + 1];
  pre[0] = 1.0;
  for (int i = 0; i < n; ++i) pre[i + 1] = pre[i] * xa[i]; /* prod_{k < i} |x_k| */
  double suf = 1.0, w = 0.0;                             /* suf = prod_{k > i} |x_k| */
  for (int i = n - 1; i >= 0; --i) {
#if ORACLE_MUTANT == 9
    w += pre[i] * suf; /* planted: row weight R_i dropped */
#else
    w += R[i] * pre[i] * suf;
#endif
    suf *= xa[i];
  }
  st->s = dd_add_d(st->s, pre[n]);
  st->w = dd_add_d(st->w, w);
}

static void ryser_dd_stats_body(const void* vctx, uint64_t s, uint64_t e, void* out) {
  const real_ctx_t* c = (const real_ctx_t*)vctx;
  const double* A = c->A;
  int n = c->n;
  dd_t x[ORACLE_NMAX];
  double R[ORACLE_NMAX], xa[ORACLE_NMAX];
  for (int i = 0; i < n; ++i) { /* Alg. 1 start state, in double-double */
    dd_t sum = DD_ZERO;
    double r = 0.0;
    for (int j = 0; j < n; ++j) {
      sum = dd_add_d(sum, A[i * n + j]);
      r += fabs(A[i * n + j]);
    }
    dd_t half = {sum.hi / 2.0, sum.lo / 2.0};
    x[i] = dd_add_d(dd_neg(half), A[i * n + (n - 1)]);
    R[i] = r;
  }
  dd_stats_t st = {DD_ZERO, DD_ZERO, DD_ZERO};
  uint64_t start = s;
  if (s == 0) { /* the g = 0 term: product of the start state */
    dd_t prod = {1.0, 0.0};
    for (int i = 0; i < n; ++i) {
      prod = dd_mul(prod, x[i]);
      xa[i] = fabs(x[i].hi);
    }
    st.p = dd_add(st.p, prod);
    stats_step(xa, R, n, &st);
    start = 1;
  }
  if (start < e) { /* Alg. 3: x at Gray_{start-1} */
    uint64_t G = oracle_gray(start - 1);
    for (int j = 0; j < n - 1; ++j)
      if ((G >> j) & 1u)
        for (int i = 0; i < n; ++i) x[i] = dd_add_d(x[i], A[i * n + j]);
  }
  for (uint64_t g = start; g < e; ++g) {
    int j = oracle_changed_bit(g);
    double sg = 2.0 * (double)((oracle_gray(g) >> j) & 1u) - 1.0;
    dd_t prod = {1.0, 0.0};
    for (int i = 0; i < n; ++i) {
      x[i] = dd_add_d(x[i], sg * A[i * n + j]);
      prod = dd_mul(prod, x[i]);
      xa[i] = fabs(x[i].hi);
    }
    st.p = (g & 1u) ? dd_add(st.p, dd_neg(prod)) : dd_add(st.p, prod);
    stats_step(xa, R, n, &st);
  }
  *(dd_stats_t*)out = st;
}

/* out = {sum hi, sum lo, S, W} for the range [g0, g1); the sum is the one of
 * oracle_ryser_dd_range (x and products in double-double). */
int oracle_ryser_dd_stats_range(const double* A, int n, uint64_t g0, uint64_t g1, int threads, double* out) {
  int rc = check_range(n, g0, g1);
  if (rc) return rc;
  real_ctx_t ctx = {A, n};
  int tau = threads < 1 ? 1 : threads;
  dd_stats_t* parts = (dd_stats_t*)calloc((size_t)tau, sizeof(dd_stats_t));
  if (!parts) return -3;
  if (run_chunks(&ctx, g0, g1, tau, ryser_dd_stats_body, parts, sizeof(dd_stats_t))) {
    free(parts);
    return -3;
  }
  dd_stats_t tot = {DD_ZERO, DD_ZERO, DD_ZERO};
  for (int t = 0; t < tau; ++t) { /* outer sum, fixed order */
    tot.p = dd_add(tot.p, parts[t].p);
    tot.s = dd_add(tot.s, parts[t].s);
    tot.w = dd_add(tot.w, parts[t].w);
  }
  free(parts);
  out[0] = tot.p.hi;
  out[1] = tot.p.lo;
  out[2] = tot.s.hi + tot.s.lo;
  out[3] = tot.w.hi + tot.w.lo;
  return 0;
}

/* complex double-double: (a + ib)(c + id) = (ac - bd) + i(ad + bc) */
typedef struct {
  dd_t re, im;
} cdd_val_t;

static cdd_val_t cdd_mul(cdd_val_t a, cdd_val_t b) {
  cdd_val_t r;
  r.re = dd_add(dd_mul(a.re, b.re), dd_neg(dd_mul(a.im, b.im)));
#if ORACLE_MUTANT == 8
  r.im = dd_add(dd_mul(a.re, b.im), dd_neg(dd_mul(a.im, b.re))); /* planted: sign of a cross term */
#else
  r.im = dd_add(dd_mul(a.re, b.im), dd_mul(a.im, b.re));
#endif
  return r;
}

typedef struct {
  dd_t pr, pi, s, w;
} cdd_stats_t;

static void ryser_cdd_body(const void* vctx, uint64_t s, uint64_t e, void* out) {
  const cplx_ctx_t* c = (const cplx_ctx_t*)vctx;
  const double* A = c->A; /* (re, im) pairs */
  int n = c->n;
  cdd_val_t x[ORACLE_NMAX];
  double R[ORACLE_NMAX], xa[ORACLE_NMAX];
  for (int i = 0; i < n; ++i) { /* x_i = a_{i,n} - (sum_j a_ij) / 2, both parts */
    dd_t sr = DD_ZERO, si = DD_ZERO;
    double r = 0.0;
    for (int j = 0; j < n; ++j) {
      sr = dd_add_d(sr, A[2 * (i * n + j)]);
      si = dd_add_d(si, A[2 * (i * n + j) + 1]);
      r += hypot(A[2 * (i * n + j)], A[2 * (i * n + j) + 1]);
    }
    dd_t half_re = {sr.hi / 2.0, sr.lo / 2.0}, half_im = {si.hi / 2.0, si.lo / 2.0};
    x[i].re = dd_add_d(dd_neg(half_re), A[2 * (i * n + n - 1)]);
    x[i].im = dd_add_d(dd_neg(half_im), A[2 * (i * n + n - 1) + 1]);
    R[i] = r;
  }
  dd_stats_t st = {DD_ZERO, DD_ZERO, DD_ZERO};
  dd_t pim = DD_ZERO;
  uint64_t start = s;
  if (s == 0) {
    cdd_val_t prod = {{1.0, 0.0}, DD_ZERO};
    for (int i = 0; i < n; ++i) {
      prod = cdd_mul(prod, x[i]);
      xa[i] = hypot(x[i].re.hi, x[i].im.hi);
    }
    st.p = dd_add(st.p, prod.re);
    pim = dd_add(pim, prod.im);
    stats_step(xa, R, n, &st);
    start = 1;
  }
  if (start < e) {
    uint64_t G = oracle_gray(start - 1);
    for (int j = 0; j < n - 1; ++j)
      if ((G >> j) & 1u)
        for (int i = 0; i < n; ++i) {
          x[i].re = dd_add_d(x[i].re, A[2 * (i * n + j)]);
          x[i].im = dd_add_d(x[i].im, A[2 * (i * n + j) + 1]);
        }
  }
  for (uint64_t g = start; g < e; ++g) {
    int j = oracle_changed_bit(g);
    double sg = 2.0 * (double)((oracle_gray(g) >> j) & 1u) - 1.0;
    cdd_val_t prod = {{1.0, 0.0}, DD_ZERO};
    for (int i = 0; i < n; ++i) {
      x[i].re = dd_add_d(x[i].re, sg * A[2 * (i * n + j)]);
      x[i].im = dd_add_d(x[i].im, sg * A[2 * (i * n + j) + 1]);
      prod = cdd_mul(prod, x[i]);
      xa[i] = hypot(x[i].re.hi, x[i].im.hi);
    }
    if (g & 1u) {
      st.p = dd_add(st.p, dd_neg(prod.re));
      pim = dd_add(pim, dd_neg(prod.im));
    } else {
      st.p = dd_add(st.p, prod.re);
      pim = dd_add(pim, prod.im);
    }
    stats_step(xa, R, n, &st);
  }
  cdd_stats_t* o = (cdd_stats_t*)out;
  o->pr = st.p;
  o->pi = pim;
  o->s = st.s;
  o->w = st.w;
}

/* out = {re hi, re lo, im hi, im lo, S, W}: the complex range sum of Alg. 1
 * with x and every product in double-double. */
int oracle_ryser_cdd_range(const double* A, int n, uint64_t g0, uint64_t g1, int threads, double* out) {
  int rc = check_range(n, g0, g1);
  if (rc) return rc;
  cplx_ctx_t ctx = {A, n};
  int tau = threads < 1 ? 1 : threads;
  cdd_stats_t* parts = (cdd_stats_t*)calloc((size_t)tau, sizeof(cdd_stats_t));
  if (!parts) return -3;
  if (run_chunks(&ctx, g0, g1, tau, ryser_cdd_body, parts, sizeof(cdd_stats_t))) {
    free(parts);
    return -3;
  }
  cdd_stats_t tot = {DD_ZERO, DD_ZERO, DD_ZERO, DD_ZERO};
  for (int t = 0; t < tau; ++t) {
    tot.pr = dd_add(tot.pr, parts[t].pr);
    tot.pi = dd_add(tot.pi, parts[t].pi);
    tot.s = dd_add(tot.s, parts[t].s);
    tot.w = dd_add(tot.w, parts[t].w);
  }
  free(parts);
  out[0] = tot.pr.hi;
  out[1] = tot.pr.lo;
  out[2] = tot.pi.hi;
  out[3] = tot.pi.lo;
  out[4] = tot.s.hi + tot.s.lo;
  out[5] = tot.w.hi + tot.w.lo;
  return 0;
}

/* ---------------------------------------------------- Alg. 2, sparse (CRS/CCS) */

typedef struct {
  int n;
  const int32_t *rptrs, *cids;
  const double* rvals;
  const int32_t *cptrs, *rids;
  const double* cvals;
} sparse_ctx_t;

static void spa_ryser_body(const void* vctx, uint64_t s, uint64_t e, void* out) {
  const sparse_ctx_t* c = (const sparse_ctx_t*)vctx;
  int n = c->n;
  double x[ORACLE_NMAX];
  for (int i = 0; i < n; ++i) { /* Alg. 2, start state from the CRS row sums */
    double sum = 0.0, a_in = 0.0;
    for (int32_t ptr = c->rptrs[i]; ptr < c->rptrs[i + 1]; ++ptr) {
      sum += c->rvals[ptr];
      if (c->cids[ptr] == n - 1) a_in = c->rvals[ptr];
    }
    x[i] = a_in - sum / 2.0;
  }
  dd_t p = DD_ZERO;
  uint64_t start = s;
  if (s == 0) { /* Alg. 2: product of the start state */
    double prod = 1.0;
    for (int i = 0; i < n; ++i) prod *= x[i];
    p = dd_add_d(p, prod);
    start = 1;
  }
  if (start < e) {
    uint64_t G = oracle_gray(start - 1);
    for (int j = 0; j < n - 1; ++j)
      if ((G >> j) & 1u)
        for (int32_t ptr = c->cptrs[j]; ptr < c->cptrs[j + 1]; ++ptr) x[c->rids[ptr]] += c->cvals[ptr];
  }
  for (uint64_t g = start; g < e; ++g) {
    int j = oracle_changed_bit(g);
    double sg = 2.0 * (double)((oracle_gray(g) >> j) & 1u) - 1.0;
    for (int32_t ptr = c->cptrs[j]; ptr < c->cptrs[j + 1]; ++ptr) { /* nonzeros of column j */
      int32_t row = c->rids[ptr];
      double val = c->cvals[ptr];
      x[row] = x[row] + sg * val;
    }
    double prod = 1.0; /* full product over all rows, as in Alg. 2 */
    for (int i = 0; i < n; ++i) prod = prod * x[i];
    p = (g & 1u) ? dd_add_d(p, -prod) : dd_add_d(p, prod);
  }
  *(dd_t*)out = p;
}

int oracle_spa_ryser_f64_range(int n, const int32_t* rptrs, const int32_t* cids, const double* rvals,
                               const int32_t* cptrs, const int32_t* rids, const double* cvals, uint64_t g0,
                               uint64_t g1, int threads, double* out) {
  int rc = check_range(n, g0, g1);
  if (rc) return rc;
  sparse_ctx_t ctx = {n, rptrs, cids, rvals, cptrs, rids, cvals};
  int tau = threads < 1 ? 1 : threads;
  dd_t* parts = (dd_t*)calloc((size_t)tau, sizeof(dd_t));
  if (!parts) return -3;
  if (run_chunks(&ctx, g0, g1, tau, spa_ryser_body, parts, sizeof(dd_t))) {
    free(parts);
    return -3;
  }
  dd_t tot = DD_ZERO;
  for (int t = 0; t < tau; ++t) tot = dd_add(tot, parts[t]);
  free(parts);
  out[0] = tot.hi;
  out[1] = tot.lo;
  return 0;
}

/* -------------------------------------------------- binary, exact integers */

typedef unsigned __int128 u128;

typedef struct {
  const uint8_t* A;
  int n;
} bin_ctx_t;

/* Eq. 2 over all S in [n] visited in Gray order (Sec. 2), every product and
 * sum reduced mod 2^128 (wrap-around is a ring homomorphism, so the result is
 * perm(A) mod 2^128). */
static void ryser_bin_plain_body(const void* vctx, uint64_t s, uint64_t e, void* out) {
  const bin_ctx_t* c = (const bin_ctx_t*)vctx;
  const uint8_t* A = c->A;
  int n = c->n;
  int64_t r[ORACLE_NMAX];
  for (int i = 0; i < n; ++i) r[i] = 0;
  uint64_t G = oracle_gray(s == 0 ? 0 : s);
  for (int j = 0; j < n; ++j)
    if ((G >> j) & 1u)
      for (int i = 0; i < n; ++i) r[i] += A[i * n + j];
  u128 acc = 0;
  for (uint64_t g = s; g < e; ++g) {
    if (g > s) {
      int j = oracle_changed_bit(g);
      int64_t sg = 2 * (int64_t)((oracle_gray(g) >> j) & 1u) - 1;
      for (int i = 0; i < n; ++i) r[i] += sg * A[i * n + j];
    }
    u128 prod = 1;
    for (int i = 0; i < n; ++i) prod *= (u128)(uint64_t)r[i]; /* r[i] >= 0 */
    int card = __builtin_popcountll(oracle_gray(g));
    acc += (card & 1) ? (u128)0 - prod : prod;
  }
  *(u128*)out = acc;
}

/* perm(A) mod 2^128 for a 0/1 matrix (entries must be 0 or 1), n <= 40. */
int oracle_ryser_bin_plain(const uint8_t* A, int n, int threads, uint64_t* out) {
  if (n < 0 || n > 40) return -1;
  if (n == 0) {
    out[0] = 1;
    out[1] = 0;
    return 0;
  }
  bin_ctx_t ctx = {A, n};
  int tau = threads < 1 ? 1 : threads;
  u128* parts = (u128*)calloc((size_t)tau, sizeof(u128));
  if (!parts) return -3;
  if (run_chunks(&ctx, 0, 1ull << n, tau, ryser_bin_plain_body, parts, sizeof(u128))) {
    free(parts);
    return -3;
  }
  u128 tot = 0;
  for (int t = 0; t < tau; ++t) tot += parts[t];
  free(parts);
  if (n & 1) tot = (u128)0 - tot; /* (-1)^n */
  out[0] = (uint64_t)tot;
  out[1] = (uint64_t)(tot >> 64);
  return 0;
}

/* Alg. 1 with the row vector doubled, x'_i = 2 a_{i,n} - r_i (exact integers):
 * sum over g in [g0, g1) of (-1)^g prod_i x'_i(g), mod 2^128.  Over the whole
 * range this equals (-1)^(n-1) 2^(n-1) perm(A) (mod 2^128). */
static void ryser_bin_range_body(const void* vctx, uint64_t s, uint64_t e, void* out) {
  const bin_ctx_t* c = (const bin_ctx_t*)vctx;
  const uint8_t* A = c->A;
  int n = c->n;
  int64_t x[ORACLE_NMAX];
  for (int i = 0; i < n; ++i) {
    int64_t sum = 0;
    for (int j = 0; j < n; ++j) sum += A[i * n + j];
    x[i] = 2 * (int64_t)A[i * n + (n - 1)] - sum;
  }
  uint64_t G = oracle_gray(s);
  for (int j = 0; j < n - 1; ++j)
    if ((G >> j) & 1u)
      for (int i = 0; i < n; ++i) x[i] += 2 * (int64_t)A[i * n + j];
  u128 acc = 0;
  for (uint64_t g = s; g < e; ++g) {
    if (g > s) {
      int j = oracle_changed_bit(g);
      int64_t sg = 2 * (int64_t)((oracle_gray(g) >> j) & 1u) - 1;
      for (int i = 0; i < n; ++i) x[i] += sg * 2 * (int64_t)A[i * n + j];
    }
    u128 prod = 1;
    for (int i = 0; i < n; ++i) prod *= (u128)(__int128)x[i];
    acc += (g & 1u) ? (u128)0 - prod : prod;
  }
  *(u128*)out = acc;
}

int oracle_ryser_bin_range(const uint8_t* A, int n, uint64_t g0, uint64_t g1, int threads, uint64_t* out) {
  int rc = check_range(n, g0, g1);
  if (rc) return rc;
  bin_ctx_t ctx = {A, n};
  int tau = threads < 1 ? 1 : threads;
  u128* parts = (u128*)calloc((size_t)tau, sizeof(u128));
  if (!parts) return -3;
  if (run_chunks(&ctx, g0, g1, tau, ryser_bin_range_body, parts, sizeof(u128))) {
    free(parts);
    return -3;
  }
  u128 tot = 0;
  for (int t = 0; t < tau; ++t) tot += parts[t];
  free(parts);
  out[0] = (uint64_t)tot;
  out[1] = (uint64_t)(tot >> 64);
  return 0;
}

/* ------------------------------------------- Eq. 1 by row-wise subset DP */
/* f_0(empty) = 1; f_i(S) = sum_{j in S} a_{i-1,j} f_{i-1}(S \ {j}) for |S| = i;
 * perm(A) = f_n({0..n-1}).  Every permutation sigma is counted once: row i-1
 * takes column j = sigma(i-1) and rows 0..i-2 take S \ {j}. */

int oracle_perm_dp_f64(const double* A, int n, double* out) {
  if (n < 0 || n > 24) return -1;
  size_t N = (size_t)1 << n;
  double* f = (double*)calloc(N, sizeof(double));
  if (!f) return -3;
  f[0] = 1.0;
  for (size_t S = 1; S < N; ++S) {
    int i = __builtin_popcountll((unsigned long long)S);
    const double* row = A + (size_t)(i - 1) * n;
    double acc = 0.0;
    for (int j = 0; j < n; ++j)
      if ((S >> j) & 1u) acc += row[j] * f[S ^ ((size_t)1 << j)];
    f[S] = acc;
  }
  out[0] = f[N - 1];
  free(f);
  return 0;
}

int oracle_perm_dp_c128(const double* A, int n, double* out) {
  if (n < 0 || n > 23) return -1;
  size_t N = (size_t)1 << n;
  double* f = (double*)calloc(2 * N, sizeof(double));
  if (!f) return -3;
  f[0] = 1.0;
  for (size_t S = 1; S < N; ++S) {
    int i = __builtin_popcountll((unsigned long long)S);
    const double* row = A + 2 * (size_t)(i - 1) * n;
    double ar = 0.0, ai = 0.0;
    for (int j = 0; j < n; ++j)
      if ((S >> j) & 1u) {
        size_t T = S ^ ((size_t)1 << j);
        double br = row[2 * j], bi = row[2 * j + 1];
        ar += br * f[2 * T] - bi * f[2 * T + 1];
        ai += br * f[2 * T + 1] + bi * f[2 * T];
      }
    f[2 * S] = ar;
    f[2 * S + 1] = ai;
  }
  out[0] = f[2 * (N - 1)];
  out[1] = f[2 * (N - 1) + 1];
  free(f);
  return 0;
}

/* exact, mod 2^128 */
int oracle_perm_dp_bin(const uint8_t* A, int n, uint64_t* out) {
  if (n < 0 || n > 22) return -1;
  size_t N = (size_t)1 << n;
  u128* f = (u128*)calloc(N, sizeof(u128));
  if (!f) return -3;
  f[0] = 1;
  for (size_t S = 1; S < N; ++S) {
    int i = __builtin_popcountll((unsigned long long)S);
    const uint8_t* row = A + (size_t)(i - 1) * n;
    u128 acc = 0;
    for (int j = 0; j < n; ++j)
      if (((S >> j) & 1u) && row[j]) acc += f[S ^ ((size_t)1 << j)];
    f[S] = acc;
  }
  out[0] = (uint64_t)f[N - 1];
  out[1] = (uint64_t)(f[N - 1] >> 64);
  free(f);
  return 0;
}
