/*
 * oracle.c -- CPU oracle for the Toeplitz tridiagonal solve T x = F,
 * T = tridiag{t_-1, t_0, t_1} (arXiv 1002.2469, eq. 1).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously-correct
 * reference the GPU path is checked against.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or constant with the CUDA library.
 *
 * Index convention: 0-based rows i = 0..N-1, row i reads
 *     t_-1 * x[i-1] + t_0 * x[i] + t_1 * x[i+1] = F[i],
 * with x[-1] = x[N] = 0.  t_-1 is the sub-diagonal (the paper's c_i of eq. 2),
 * t_1 the super-diagonal (the paper's a_i).
 *
 * Contents
 *   oracle_thomas_f64       sequential Thomas algorithm (no pivoting), FP64
 *                           -- the "sequential version of the Thomas
 *                           algorithm" the paper uses for eq. 7 (Sec. 2.2).
 *   oracle_thomas_q         the same in binary128 (arbiter).
 *   oracle_thomas_tridiag   Thomas for a general tridiagonal matrix (three arrays),
 *                           e.g. the quasi-Toeplitz matrices of eq. 21.
 *   oracle_thomas_batched   one Thomas per system over a pthread pool.
 *   oracle_adjoint_f64      lambda = T^-T w and dL/dt for L = <w, x>.
 *   oracle_dich_eq15        the paper's Dichotomy formulas written out for a
 *                           given block partition: Green rows by eq. 9,
 *                           exterior vectors by eq. 10-12, beta by eq. 16,
 *                           first/last values by eq. 15, interiors by eq. 7.
 *   oracle_dich_levels      the same interface values by the level-by-level
 *                           dichotomy process of eq. 17-19 (Sec. 2.4).
 * Every function returns 0 on success, nonzero on a zero pivot / bad input.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

/* Planted-mistake builds: a test compiles this file with -DORACLE_MUTANT=k (k = 1..6) to
 * check that the pins catch each mistake.  The normal build uses 0 (no mistake). */
#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

#if defined(__aarch64__) && (__LDBL_MANT_DIG__ == 113)
typedef long double q128_t;          /* IEEE binary128 on aarch64 Linux */
#else
typedef __float128 q128_t;           /* GCC binary128 on x86_64 */
#endif

/* ------------------------------------------------------------------ */
/* Thomas algorithm (forward elimination, back substitution).          */
/* Works for a general tridiagonal matrix given as three arrays; the   */
/* Toeplitz entry points pass constant coefficients through it.        */
/* ------------------------------------------------------------------ */
static int thomas_general(int64_t n, const double* sub, const double* dia,
                          const double* sup, const double* f, double* x) {
  if (n <= 0) return 0;
  double* cp = (double*)malloc(sizeof(double) * (size_t)n);
  double* dp = (double*)malloc(sizeof(double) * (size_t)n);
  if (!cp || !dp) { free(cp); free(dp); return 2; }
  double m = dia[0];
  if (m == 0.0) { free(cp); free(dp); return 1; }
  cp[0] = sup[0] / m;
  dp[0] = f[0] / m;
  for (int64_t i = 1; i < n; ++i) {
    m = dia[i] - sub[i] * cp[i - 1];
    if (m == 0.0) { free(cp); free(dp); return 1; }
    cp[i] = sup[i] / m;
    dp[i] = (f[i] - sub[i] * dp[i - 1]) / m;
  }
  x[n - 1] = dp[n - 1];
  for (int64_t i = n - 2; i >= 0; --i) x[i] = dp[i] - cp[i] * x[i + 1];
  free(cp);
  free(dp);
  return 0;
}

/* General tridiagonal solve, FP64: row i reads sub[i] x[i-1] + dia[i] x[i] + sup[i] x[i+1]
 * = f[i] (sub[0] and sup[n-1] unused).  Serves the quasi-Toeplitz matrices of eq. 21 (t_0
 * replaced by t_0 + psi in the first row and t_0 + chi in the last). */
int oracle_thomas_tridiag(int64_t n, const double* sub, const double* dia, const double* sup,
                          const double* f, double* x) {
  if (n < 0) return 3;
  return thomas_general(n, sub, dia, sup, f, x);
}

/* Toeplitz solve, FP64. */
int oracle_thomas_f64(int64_t N, double tm1, double t0, double tp1,
                      const double* F, double* x) {
  if (N < 0) return 3;
  if (N == 0) return 0;
  double* cp = (double*)malloc(sizeof(double) * (size_t)N);
  double* dp = (double*)malloc(sizeof(double) * (size_t)N);
  if (!cp || !dp) { free(cp); free(dp); return 2; }
  double m = t0;
  if (m == 0.0) { free(cp); free(dp); return 1; }
  cp[0] = tp1 / m;
  dp[0] = F[0] / m;
  for (int64_t i = 1; i < N; ++i) {
#if ORACLE_MUTANT == 4
    m = t0 + tm1 * cp[i - 1];                 /* planted: wrong sign */
#else
    m = t0 - tm1 * cp[i - 1];
#endif
    if (m == 0.0) { free(cp); free(dp); return 1; }
#if ORACLE_MUTANT == 3
    cp[i] = tp1 / t0;                         /* planted: stale pivot */
#else
    cp[i] = tp1 / m;
#endif
#if ORACLE_MUTANT == 1
    dp[i] = (F[i] - tp1 * dp[i - 1]) / m;     /* planted: transposed operand */
#else
    dp[i] = (F[i] - tm1 * dp[i - 1]) / m;
#endif
  }
  x[N - 1] = dp[N - 1];
#if ORACLE_MUTANT == 2
  for (int64_t i = N - 2; i >= 0; --i) x[i] = dp[i];   /* planted: dropped term */
#else
  for (int64_t i = N - 2; i >= 0; --i) x[i] = dp[i] - cp[i] * x[i + 1];
#endif
  free(cp);
  free(dp);
  return 0;
}

/* Toeplitz solve carried out entirely in binary128; result rounded to FP64. */
int oracle_thomas_q(int64_t N, double tm1, double t0, double tp1,
                    const double* F, double* x) {
  if (N < 0) return 3;
  if (N == 0) return 0;
  q128_t* cp = (q128_t*)malloc(sizeof(q128_t) * (size_t)N);
  q128_t* dp = (q128_t*)malloc(sizeof(q128_t) * (size_t)N);
  if (!cp || !dp) { free(cp); free(dp); return 2; }
  const q128_t a = tm1, b = t0, c = tp1;
  q128_t m = b;
  if (m == 0) { free(cp); free(dp); return 1; }
  cp[0] = c / m;
  dp[0] = (q128_t)F[0] / m;
  for (int64_t i = 1; i < N; ++i) {
    m = b - a * cp[i - 1];
    if (m == 0) { free(cp); free(dp); return 1; }
    cp[i] = c / m;
    dp[i] = ((q128_t)F[i] - a * dp[i - 1]) / m;
  }
  q128_t xn = dp[N - 1];
  x[N - 1] = (double)xn;
  for (int64_t i = N - 2; i >= 0; --i) {
    xn = dp[i] - cp[i] * xn;
    x[i] = (double)xn;
  }
  free(cp);
  free(dp);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Batched: systems s = 0..nsys-1 stored back to back, system s at     */
/* F[off[s] .. off[s]+N[s]).  Each system is one sequential Thomas     */
/* solve; systems are spread over nthreads POSIX threads.              */
/* ------------------------------------------------------------------ */
typedef struct {
  int64_t nsys;
  const int64_t* N;
  const int64_t* off;
  const double *tm1, *t0, *tp1, *F;
  double* x;
  int64_t next;          /* shared work counter */
  pthread_mutex_t mu;
  int status;
} batch_job;

static void* batch_worker(void* arg) {
  batch_job* j = (batch_job*)arg;
  for (;;) {
    pthread_mutex_lock(&j->mu);
    int64_t s = j->next++;
    pthread_mutex_unlock(&j->mu);
    if (s >= j->nsys) break;
    int rc = oracle_thomas_f64(j->N[s], j->tm1[s], j->t0[s], j->tp1[s],
                               j->F + j->off[s], j->x + j->off[s]);
    if (rc) {
      pthread_mutex_lock(&j->mu);
      j->status = rc;
      pthread_mutex_unlock(&j->mu);
    }
  }
  return NULL;
}

int oracle_thomas_batched(int64_t nsys, const int64_t* N, const int64_t* off,
                          const double* tm1, const double* t0, const double* tp1,
                          const double* F, double* x, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 1024) nthreads = 1024;
  batch_job j;
  j.nsys = nsys; j.N = N; j.off = off; j.tm1 = tm1; j.t0 = t0; j.tp1 = tp1;
  j.F = F; j.x = x; j.next = 0; j.status = 0;
  pthread_mutex_init(&j.mu, NULL);
  pthread_t th[1024];
  int started = 0;
  for (int i = 0; i < nthreads; ++i) {
    if (pthread_create(&th[i], NULL, batch_worker, &j) != 0) break;
    ++started;
  }
  if (started == 0) batch_worker(&j);
  for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
  pthread_mutex_destroy(&j.mu);
  return j.status;
}

/* ------------------------------------------------------------------ */
/* Adjoint of L = <w, x>, x = T^-1 F:                                  */
/*   lambda = T^-T w  (T^T = tridiag{t_1, t_0, t_-1}),                 */
/*   dL/dF = lambda, dL/dT = -lambda x^T, so                           */
/*   dL/dt_-1 = -sum_{i>=1} lambda_i x_{i-1},                          */
/*   dL/dt_0  = -sum_i      lambda_i x_i,                              */
/*   dL/dt_1  = -sum_{i<=N-2} lambda_i x_{i+1}.                        */
/* gt[0..2] = (dL/dt_-1, dL/dt_0, dL/dt_1).                            */
/* ------------------------------------------------------------------ */
int oracle_adjoint_f64(int64_t N, double tm1, double t0, double tp1,
                       const double* w, const double* x, double* lam, double* gt) {
#if ORACLE_MUTANT == 5
  int rc = oracle_thomas_f64(N, tm1, t0, tp1, w, lam);   /* planted: T instead of T^T */
#else
  int rc = oracle_thomas_f64(N, tp1, t0, tm1, w, lam);
#endif
  if (rc) return rc;
  double gm = 0.0, g0 = 0.0, gp = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    g0 -= lam[i] * x[i];
#if ORACLE_MUTANT == 6
    if (i + 1 < N) gm -= lam[i] * x[i + 1];             /* planted: shifted the wrong way */
    if (i >= 1) gp -= lam[i] * x[i - 1];
#else
    if (i >= 1) gm -= lam[i] * x[i - 1];
    if (i + 1 < N) gp -= lam[i] * x[i + 1];
#endif
  }
  gt[0] = gm; gt[1] = g0; gt[2] = gp;
  return 0;
}

/* ------------------------------------------------------------------ */
/* The Dichotomy formulas, written out for a block partition.           */
/*                                                                      */
/* Blocks m = 0..P-1; block m holds rows [s_m, e_m] with s_0 = 0,        */
/* e_{P-1} = N-1, s_{m+1} = e_m + 1 and e_m - s_m >= 1 (size >= 2, as    */
/* Sec. 2.1 requires).  starts[m] = s_m.                                 */
/*                                                                      */
/* Preliminary step (Sec. 2.3):                                         */
/*   G^L_m : A^T G = e_{s_m},  G^R_m : A^T G = e_{e_m}      (eq. 9)      */
/*   Z^L_m : on rows 0..s_m-1, {A} z = -a_{s_m-1} e^L, Z^L_m(s_m) = 1    */
/*   Z^R_m : on rows e_m+1..N-1, {A} z = -c_{e_m+1} e^R, Z^R_m(e_m) = 1  */
/*                                                          (eq. 10-12)  */
/* Dichotomy process:                                                   */
/*   beta^{L,R}_m = sum_{j in block m} F_j G^{L,R}_m(j)          (eq. 16) */
/*   x_{s_m} = sum_{j<m} beta^R_j Z^R_j(s_m) + sum_{j>=m} beta^L_j Z^L_j(s_m)
/*   x_{e_m} = sum_{j<=m} beta^R_j Z^R_j(e_m) + sum_{j>m} beta^L_j Z^L_j(e_m)
/*                                                               (eq. 15) */
/*   interior rows s_m+1..e_m-1 by eq. 7 with Thomas.                    */
/* Outputs (any may be NULL except x):                                  */
/*   x[N], beta_L[P], beta_R[P], xs[P] = x_{s_m}, xe[P] = x_{e_m}.         */
/* ------------------------------------------------------------------ */
typedef struct {
  int64_t N, P;
  const int64_t* s;       /* block starts */
  int64_t* e;             /* block ends */
  double *sub, *dia, *sup;/* full matrix diagonals, length N */
  double* GL;             /* P x N */
  double* GR;             /* P x N */
  double* ZL;             /* P x N, valid on 0..s_m */
  double* ZR;             /* P x N, valid on e_m..N-1 */
} dich_pre;

static void dich_pre_free(dich_pre* d) {
  free(d->e); free(d->sub); free(d->dia); free(d->sup);
  free(d->GL); free(d->GR); free(d->ZL); free(d->ZR);
}

static int dich_pre_build(int64_t N, double tm1, double t0, double tp1,
                          int64_t P, const int64_t* starts, dich_pre* d) {
  memset(d, 0, sizeof(*d));
  if (N < 2 || P < 1 || starts[0] != 0) return 3;
  for (int64_t m = 0; m < P; ++m) {
    int64_t e = (m + 1 < P) ? starts[m + 1] - 1 : N - 1;
    if (e - starts[m] < 1) return 3;      /* every sub-vector needs size >= 2 */
  }
  d->N = N; d->P = P; d->s = starts;
  d->e = (int64_t*)malloc(sizeof(int64_t) * (size_t)P);
  d->sub = (double*)malloc(sizeof(double) * (size_t)N);
  d->dia = (double*)malloc(sizeof(double) * (size_t)N);
  d->sup = (double*)malloc(sizeof(double) * (size_t)N);
  d->GL = (double*)calloc((size_t)(P * N), sizeof(double));
  d->GR = (double*)calloc((size_t)(P * N), sizeof(double));
  d->ZL = (double*)calloc((size_t)(P * N), sizeof(double));
  d->ZR = (double*)calloc((size_t)(P * N), sizeof(double));
  if (!d->e || !d->sub || !d->dia || !d->sup || !d->GL || !d->GR || !d->ZL || !d->ZR) {
    dich_pre_free(d);
    return 2;
  }
  for (int64_t m = 0; m < P; ++m) d->e[m] = (m + 1 < P) ? starts[m + 1] - 1 : N - 1;
  for (int64_t i = 0; i < N; ++i) {
    d->sub[i] = (i > 0) ? tm1 : 0.0;       /* c_i */
    d->dia[i] = t0;                        /* b_i */
    d->sup[i] = (i + 1 < N) ? tp1 : 0.0;   /* a_i */
  }
  /* A^T has sub-diagonal a_{i-1} and super-diagonal c_{i+1}. */
  double* tsub = (double*)malloc(sizeof(double) * (size_t)N);
  double* tsup = (double*)malloc(sizeof(double) * (size_t)N);
  double* rhs = (double*)calloc((size_t)N, sizeof(double));
  if (!tsub || !tsup || !rhs) { free(tsub); free(tsup); free(rhs); dich_pre_free(d); return 2; }
  for (int64_t i = 0; i < N; ++i) {
    tsub[i] = (i > 0) ? d->sup[i - 1] : 0.0;
    tsup[i] = (i + 1 < N) ? d->sub[i + 1] : 0.0;
  }
  int rc = 0;
  for (int64_t m = 0; m < P && !rc; ++m) {
    /* eq. 9 */
    memset(rhs, 0, sizeof(double) * (size_t)N);
    rhs[d->s[m]] = 1.0;
    rc |= thomas_general(N, tsub, d->dia, tsup, rhs, d->GL + m * N);
    rhs[d->s[m]] = 0.0;
    rhs[d->e[m]] = 1.0;
    rc |= thomas_general(N, tsub, d->dia, tsup, rhs, d->GR + m * N);
    rhs[d->e[m]] = 0.0;
    /* eq. 11: rows 0..s-1 of A with RHS -a_{s-1} in the last row */
    int64_t s = d->s[m];
    d->ZL[m * N + s] = 1.0;
    if (s > 0) {
      memset(rhs, 0, sizeof(double) * (size_t)N);
      rhs[s - 1] = -d->sup[s - 1];
      rc |= thomas_general(s, d->sub, d->dia, d->sup, rhs, d->ZL + m * N);
    }
    /* eq. 12: rows e+1..N-1 of A with RHS -c_{e+1} in the first row */
    int64_t e = d->e[m];
    d->ZR[m * N + e] = 1.0;
    if (e + 1 < N) {
      int64_t len = N - 1 - e;
      memset(rhs, 0, sizeof(double) * (size_t)N);
      rhs[0] = -d->sub[e + 1];
      rc |= thomas_general(len, d->sub + e + 1, d->dia + e + 1, d->sup + e + 1, rhs,
                           d->ZR + m * N + e + 1);
    }
  }
  free(tsub); free(tsup); free(rhs);
  if (rc) { dich_pre_free(d); return 1; }
  return 0;
}

/* eq. 7: interior rows s+1..e-1 with x_s, x_e known. */
static int dich_interior(const dich_pre* d, const double* F, int64_t m, double* x) {
  int64_t s = d->s[m], e = d->e[m];
  int64_t len = e - s - 1;
  if (len <= 0) return 0;
  double* rhs = (double*)malloc(sizeof(double) * (size_t)len);
  if (!rhs) return 2;
  for (int64_t k = 0; k < len; ++k) rhs[k] = F[s + 1 + k];
  rhs[0] -= d->sub[s + 1] * x[s];          /* c_{m_L+1} x_{m_L} */
  rhs[len - 1] -= d->sup[e - 1] * x[e];    /* a_{m_R-1} x_{m_R} */
  int rc = thomas_general(len, d->sub + s + 1, d->dia + s + 1, d->sup + s + 1, rhs, x + s + 1);
  free(rhs);
  return rc;
}

static void dich_betas(const dich_pre* d, const double* F, double* bL, double* bR) {
  for (int64_t m = 0; m < d->P; ++m) {
    double l = 0.0, r = 0.0;
    for (int64_t j = d->s[m]; j <= d->e[m]; ++j) {
      l += F[j] * d->GL[m * d->N + j];
      r += F[j] * d->GR[m * d->N + j];
    }
    bL[m] = l;
    bR[m] = r;
  }
}

int oracle_dich_eq15(int64_t N, double tm1, double t0, double tp1, const double* F,
                     int64_t P, const int64_t* starts, double* x,
                     double* beta_L, double* beta_R, double* xs, double* xe) {
  dich_pre d;
  int rc = dich_pre_build(N, tm1, t0, tp1, P, starts, &d);
  if (rc) return rc;
  double* bL = (double*)malloc(sizeof(double) * (size_t)P);
  double* bR = (double*)malloc(sizeof(double) * (size_t)P);
  if (!bL || !bR) { free(bL); free(bR); dich_pre_free(&d); return 2; }
  dich_betas(&d, F, bL, bR);
  for (int64_t m = 0; m < P; ++m) {
    int64_t s = d.s[m], e = d.e[m];
    double vs = 0.0, ve = 0.0;
    for (int64_t j = 0; j < m; ++j) vs += bR[j] * d.ZR[j * N + s];
    for (int64_t j = m; j < P; ++j) vs += bL[j] * d.ZL[j * N + s];
    for (int64_t j = 0; j <= m; ++j) ve += bR[j] * d.ZR[j * N + e];
    for (int64_t j = m + 1; j < P; ++j) ve += bL[j] * d.ZL[j * N + e];
    x[s] = vs;
    x[e] = ve;
  }
  for (int64_t m = 0; m < P && !rc; ++m) rc = dich_interior(&d, F, m, x);
  if (beta_L) memcpy(beta_L, bL, sizeof(double) * (size_t)P);
  if (beta_R) memcpy(beta_R, bR, sizeof(double) * (size_t)P);
  if (xs) for (int64_t m = 0; m < P; ++m) xs[m] = x[d.s[m]];
  if (xe) for (int64_t m = 0; m < P; ++m) xe[m] = x[d.e[m]];
  free(bL); free(bR);
  dich_pre_free(&d);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Level-by-level dichotomy process (Sec. 2.4, eq. 17-19).             */
/* A group [lo, hi] of blocks whose beta-hat values already carry all  */
/* contributions from outside the group is split at its middle block m:*/
/*   xi^R = sum_{j=lo}^{m-1} bR_j Z^R_j(s_m),                           */
/*   xi^L = sum_{j=m+1}^{hi} bL_j Z^L_j(e_m)                  (eq. 17)  */
/*   x_{s_m} = xi^R + xi^L G^L_m(e_m)/G^R_m(e_m) + bL_m,                */
/*   x_{e_m} = xi^R G^R_m(s_m)/G^L_m(s_m) + xi^L + bR_m       (eq. 18)  */
/*   delta^L = (x_{s_m} - xi^R) Z^L_m(s_m - 1)  -> block m-1,           */
/*   delta^R = (x_{e_m} - xi^L) Z^R_m(e_m + 1)  -> block m+1,           */
/*   bR_{m-1} += delta^L, bL_{m-1} += delta^L G^L_{m-1}(e_{m-1})/G^R_{m-1}(e_{m-1}),
/*   bL_{m+1} += delta^R, bR_{m+1} += delta^R G^R_{m+1}(s_{m+1})/G^L_{m+1}(s_{m+1})
/*                                                            (eq. 19)  */
/* then the two sub-groups are processed the same way.                 */
/* ------------------------------------------------------------------ */
static void dich_level(const dich_pre* d, double* bL, double* bR, int64_t lo, int64_t hi,
                       double* xs, double* xe, int depth, int* max_depth) {
  if (lo > hi) return;
  if (depth > *max_depth) *max_depth = depth;
  const int64_t N = d->N;
  int64_t m = lo + (hi - lo) / 2;
  int64_t s = d->s[m], e = d->e[m];
  double xiR = 0.0, xiL = 0.0;
  for (int64_t j = lo; j < m; ++j) xiR += bR[j] * d->ZR[j * N + s];
  for (int64_t j = m + 1; j <= hi; ++j) xiL += bL[j] * d->ZL[j * N + e];
  const double* gl = d->GL + m * N;
  const double* gr = d->GR + m * N;
  double vs = xiR + xiL * (gl[e] / gr[e]) + bL[m];
  double ve = xiR * (gr[s] / gl[s]) + xiL + bR[m];
  xs[m] = vs;
  xe[m] = ve;
  if (m - 1 >= lo) {
    double dL = (xiL * (gl[e] / gr[e]) + bL[m]) * d->ZL[m * N + s - 1];
    int64_t q = m - 1;
    int64_t tR = d->e[q];
    bR[q] += dL;
    bL[q] += dL * (d->GL[q * N + tR] / d->GR[q * N + tR]);
  }
  if (m + 1 <= hi) {
    double dR = (xiR * (gr[s] / gl[s]) + bR[m]) * d->ZR[m * N + e + 1];
    int64_t q = m + 1;
    int64_t qL = d->s[q];
    bL[q] += dR;
    bR[q] += dR * (d->GR[q * N + qL] / d->GL[q * N + qL]);
  }
  dich_level(d, bL, bR, lo, m - 1, xs, xe, depth + 1, max_depth);
  dich_level(d, bL, bR, m + 1, hi, xs, xe, depth + 1, max_depth);
}

int oracle_dich_levels(int64_t N, double tm1, double t0, double tp1, const double* F,
                       int64_t P, const int64_t* starts, double* x, int* levels) {
  dich_pre d;
  int rc = dich_pre_build(N, tm1, t0, tp1, P, starts, &d);
  if (rc) return rc;
  double* bL = (double*)malloc(sizeof(double) * (size_t)P);
  double* bR = (double*)malloc(sizeof(double) * (size_t)P);
  double* xs = (double*)malloc(sizeof(double) * (size_t)P);
  double* xe = (double*)malloc(sizeof(double) * (size_t)P);
  if (!bL || !bR || !xs || !xe) { free(bL); free(bR); free(xs); free(xe); dich_pre_free(&d); return 2; }
  dich_betas(&d, F, bL, bR);
  int maxd = 0;
  dich_level(&d, bL, bR, 0, P - 1, xs, xe, 1, &maxd);
  for (int64_t m = 0; m < P; ++m) { x[d.s[m]] = xs[m]; x[d.e[m]] = xe[m]; }
  for (int64_t m = 0; m < P && !rc; ++m) rc = dich_interior(&d, F, m, x);
  if (levels) *levels = maxd;
  free(bL); free(bR); free(xs); free(xe);
  dich_pre_free(&d);
  return rc;
}

/* The preliminary vectors themselves, for pinning against closed forms:
 * out_GL/out_GR/out_ZL/out_ZR are P x N row-major (entries outside the
 * ranges named above are 0). */
int oracle_dich_prelim(int64_t N, double tm1, double t0, double tp1,
                       int64_t P, const int64_t* starts,
                       double* out_GL, double* out_GR, double* out_ZL, double* out_ZR) {
  dich_pre d;
  int rc = dich_pre_build(N, tm1, t0, tp1, P, starts, &d);
  if (rc) return rc;
  size_t bytes = sizeof(double) * (size_t)(P * N);
  if (out_GL) memcpy(out_GL, d.GL, bytes);
  if (out_GR) memcpy(out_GR, d.GR, bytes);
  if (out_ZL) memcpy(out_ZL, d.ZL, bytes);
  if (out_ZR) memcpy(out_ZR, d.ZR, bytes);
  dich_pre_free(&d);
  return 0;
}
