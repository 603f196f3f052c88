/*
 * aa_oracle.c -- plain, slow, obviously-correct FP64 CPU oracle for
 * low-synchronization Anderson acceleration (Lockhart, Gardner, Woodward,
 * Thomas, Olson, "Performance of Low Synchronization Orthogonalization
 * Methods in Anderson Accelerated Fixed Point Solvers", arXiv 2110.09667).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this code.  It shares nothing with
 * the CUDA path: no headers, helpers, tables or constants.
 *
 * Conventions (Sec. 3 of the paper): 0-based indices, inclusive slices,
 * columns of F ordered oldest -> newest.  Every sum is a sequential
 * left-to-right loop in double precision; the file is compiled with
 * -ffp-contract=off so that no multiply-add is fused behind our back.
 *
 * Readings where the paper is silent or garbled:
 *  - QRDelete (Sec. 2.1, Sec. 3.2 text): textbook Givens column deletion.
 *  - ICWY after a delete (Sec. 3.2): the strictly-lower part of T is
 *    recomputed from the rotated Q in one reduction.
 *  - ICWY stores the unit-lower I + L and applies its inverse by forward
 *    substitution (Algorithm 4).
 *  - DCGS-2 (Algorithm 6): the projection of q_{m_i-2} uses all columns
 *    0..m_i-3; the reorthogonalisation runs only when m_i > 3 (configurable);
 *    R_{0:m_i-3,m_i-2} += s literally (an option scales s by R_{m_i-2,m_i-2});
 *    the reorthogonalised column is not renormalised.
 *  - The least-squares right-hand side Q^T f_i is one extra reduction that
 *    the paper's synchronization tallies do not count (Algorithm 2).
 *  - Breakdown: if the new column's norm rho <= 1e-14 * ||Delta f|| (or is
 *    not a positive finite number) the column is not added and the whole
 *    history is cleared; that step then returns x_{i+1} = G(x_i).
 *  - Optional storage rounding emulates FP32 or BF16 storage of Q and dG.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Two builds of this one file.  The reference build (plain gcc) runs every
 * loop and every sum sequentially, as described above.  The timed build
 * (gcc -fopenmp) runs the element-wise loops in parallel with static
 * schedules, which changes no arithmetic, and each dot product as fixed
 * contiguous chunks (one per thread) whose partial sums are added in chunk
 * order: the same result for the same thread count, and with one thread
 * exactly the reference build's sum. */
#ifdef _OPENMP
#define ORA_PAR_FOR _Pragma("omp parallel for schedule(static)")
#else
#define ORA_PAR_FOR
#endif

#define ORA_MGS 0
#define ORA_ICWY 1
#define ORA_CGS2 2
#define ORA_DCGS2 3

#define ORA_OK 0
#define ORA_NOTCONVERGED 1
#define ORA_BREAKDOWN 2
#define ORA_EINVAL -1
#define ORA_ENOMEM -2
#define ORA_ENONFINITE -3

typedef struct ora_ctx {
  int64_t n;
  int m;
  int orth;
  int dcgs2_min_mi;   /* reorthogonalise in DCGS-2 only when m_i > this */
  int dcgs2_scaled;   /* 0: R += s (literal); 1: R += R_{kk} * s */
  int store_round;    /* 0: none; 1: round stored Q/dG entries to fp32; 2: bf16 */
  double breakdown_tol;
  double *Q;          /* n x m, column j at Q + j*n */
  double *R;          /* m x m row-major */
  double *T;          /* m x m row-major, unit lower (ICWY) */
  double *dG;         /* n x m ring: logical column j at slot (head + j) % m */
  double *f_prev, *g_prev, *v, *y, *f;
  int c;              /* columns held in the QR factorization */
  int head;           /* ring head of dG */
  int64_t it;         /* steps taken */
  long long syncs_qr; /* reductions counted as in the paper's tallies */
  long long syncs_lsq;/* reductions for Q^T f_i (not counted by the paper) */
  long long syncs_other; /* norms for breakdown / stopping tests */
  int last_status;
} ora_ctx;

/* ---------------------------------------------------------------- helpers */

static double dot_seq(const double *a, const double *b, int64_t n) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

static double dot(const double *a, const double *b, int64_t n) {
#ifdef _OPENMP
  enum { MAXCH = 1024 };
  int nch = omp_get_max_threads();
  if (nch > MAXCH) nch = MAXCH;
  if (nch > 1 && n >= 4096) {
    double part[MAXCH];
#pragma omp parallel for schedule(static, 1)
    for (int ch = 0; ch < nch; ++ch) {
      const int64_t lo = n * ch / nch, hi = n * (ch + 1) / nch;
      part[ch] = dot_seq(a + lo, b + lo, hi - lo);
    }
    double s = 0.0;
    for (int ch = 0; ch < nch; ++ch) s += part[ch];
    return s;
  }
#endif
  return dot_seq(a, b, n);
}

static double nrm2(const double *a, int64_t n) { return sqrt(dot(a, a, n)); }

static double *col(double *A, int64_t n, int j) { return A + (int64_t)j * n; }

/* Round-to-nearest-even to bfloat16, returned as a double. */
static double round_bf16(double x) {
  float f = (float)x;
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return (double)f; /* inf / nan */
  uint32_t lsb = (u >> 16) & 1u;
  u += 0x7fffu + lsb;
  u &= 0xffff0000u;
  memcpy(&f, &u, 4);
  return (double)f;
}

static void store_round_vec(ora_ctx *c, double *a) {
  if (c->store_round == 1) {
    ORA_PAR_FOR
    for (int64_t i = 0; i < c->n; ++i) a[i] = (double)(float)a[i];
  } else if (c->store_round == 2) {
    ORA_PAR_FOR
    for (int64_t i = 0; i < c->n; ++i) a[i] = round_bf16(a[i]);
  }
}

/* Threads of the timed (OpenMP) build; returns the count in effect (1 in
 * the reference build). */
int ora_set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
  return omp_get_max_threads();
#else
  (void)nthreads;
  return 1;
#endif
}

/* One stored history entry as the precision form keeps it: mode 1 FP32
 * (round to nearest), mode 2 BF16 (FP64 -> FP32 round to nearest, then
 * FP32 -> BF16 round to nearest even); mode 0 leaves it FP64.  Exported so
 * that the rounding itself can be pinned against literal bit patterns. */
double ora_store_round(int mode, double x) {
  if (mode == 1) return (double)(float)x;
  if (mode == 2) return round_bf16(x);
  return x;
}

/* ------------------------------------------------------------- lifecycle */

ora_ctx *ora_create(int64_t n, int m, int orth) {
  if (n < 1 || m < 1 || orth < 0 || orth > 3) return NULL;
  ora_ctx *c = (ora_ctx *)calloc(1, sizeof(ora_ctx));
  if (!c) return NULL;
  c->n = n;
  c->m = m;
  c->orth = orth;
  c->dcgs2_min_mi = 3;
  c->breakdown_tol = 1e-14;
  size_t nm = (size_t)n * (size_t)m;
  c->Q = (double *)calloc(nm, sizeof(double));
  c->dG = (double *)calloc(nm, sizeof(double));
  c->R = (double *)calloc((size_t)m * m, sizeof(double));
  c->T = (double *)calloc((size_t)m * m, sizeof(double));
  c->f_prev = (double *)calloc((size_t)n, sizeof(double));
  c->g_prev = (double *)calloc((size_t)n, sizeof(double));
  c->v = (double *)calloc((size_t)n, sizeof(double));
  c->y = (double *)calloc((size_t)n, sizeof(double));
  c->f = (double *)calloc((size_t)n, sizeof(double));
  if (!c->Q || !c->dG || !c->R || !c->T || !c->f_prev || !c->g_prev || !c->v || !c->y || !c->f) {
    free(c->Q); free(c->dG); free(c->R); free(c->T); free(c->f_prev); free(c->g_prev);
    free(c->v); free(c->y); free(c->f); free(c);
    return NULL;
  }
  return c;
}

void ora_destroy(ora_ctx *c) {
  if (!c) return;
  free(c->Q); free(c->dG); free(c->R); free(c->T); free(c->f_prev); free(c->g_prev);
  free(c->v); free(c->y); free(c->f);
  free(c);
}

/* key: 0 dcgs2_min_mi, 1 dcgs2_scaled, 2 store_round, 3 breakdown_tol */
int ora_set_option(ora_ctx *c, int key, double val) {
  switch (key) {
    case 0: c->dcgs2_min_mi = (int)val; return ORA_OK;
    case 1: c->dcgs2_scaled = (int)val; return ORA_OK;
    case 2: c->store_round = (int)val; return ORA_OK;
    case 3: c->breakdown_tol = val; return ORA_OK;
    default: return ORA_EINVAL;
  }
}

void ora_reset(ora_ctx *c) {
  c->c = 0;
  c->head = 0;
  c->it = 0;
  memset(c->R, 0, sizeof(double) * (size_t)c->m * c->m);
  memset(c->T, 0, sizeof(double) * (size_t)c->m * c->m);
}

void ora_counters(const ora_ctx *c, long long *out4) {
  out4[0] = c->syncs_qr;
  out4[1] = c->syncs_lsq;
  out4[2] = c->syncs_other;
  out4[3] = c->c;
}

/* ------------------------------------------------------------ QRDelete */

/* Remove the oldest column of Q R = F with Givens rotations (textbook column
 * deletion; the paper states only that it uses Givens rotations and needs no
 * reduction).  Drop column 0 of R, leaving an upper-Hessenberg m x (m-1)
 * matrix H; for j = 0..m-2 rotate rows j, j+1 of H to zero H[j+1][j] and
 * apply the same rotation to columns j, j+1 of Q.  Keep the leading
 * (m-1) x (m-1) block of H and the first m-1 columns of Q. */
static void qr_delete(ora_ctx *c) {
  const int m = c->c;
  const int64_t n = c->n;
  double *R = c->R;
  const int M = c->m;
  /* H[j][l] = R[j][l+1] */
  for (int j = 0; j < m; ++j) {
    for (int l = 0; l < m - 1; ++l) R[j * M + l] = R[j * M + l + 1];
    R[j * M + (m - 1)] = 0.0;
  }
  for (int j = 0; j < m - 1; ++j) {
    double a = R[j * M + j];
    double b = R[(j + 1) * M + j];
    double rho = hypot(a, b);
    double cs = 1.0, sn = 0.0;
    if (rho != 0.0) {
      cs = a / rho;
      sn = b / rho;
    }
    for (int l = j; l < m - 1; ++l) {
      double hj = R[j * M + l];
      double hj1 = R[(j + 1) * M + l];
      R[j * M + l] = cs * hj + sn * hj1;
      R[(j + 1) * M + l] = -sn * hj + cs * hj1;
    }
    R[(j + 1) * M + j] = 0.0;
    double *qj = col(c->Q, n, j);
    double *qj1 = col(c->Q, n, j + 1);
    ORA_PAR_FOR
    for (int64_t i = 0; i < n; ++i) {
      double a_i = qj[i];
      double b_i = qj1[i];
      qj[i] = cs * a_i + sn * b_i;
      qj1[i] = -sn * a_i + cs * b_i;
    }
  }
  for (int l = 0; l < M; ++l) R[(m - 1) * M + l] = 0.0;
  for (int j = 0; j < m - 1; ++j) store_round_vec(c, col(c->Q, n, j));
  c->c = m - 1;
}

/* ICWY after a delete (Sec. 3.2): with T stored explicitly, the rotated Q
 * needs its strictly-lower Gram recomputed -- one reduction.  Rows
 * 1..k-2 are refreshed here; row k-1 is the delayed row that the next
 * QRAdd_ICWY computes itself. */
static void icwy_refresh_T(ora_ctx *c) {
  const int k = c->c;
  const int M = c->m;
  for (int j = 0; j < k; ++j) {
    for (int l = 0; l < M; ++l) c->T[j * M + l] = 0.0;
    c->T[j * M + j] = 1.0;
  }
  for (int j = 1; j <= k - 2; ++j)
    for (int l = 0; l < j; ++l)
      c->T[j * M + l] = dot(col(c->Q, c->n, l), col(c->Q, c->n, j), c->n);
  c->syncs_qr += 1;
}

/* -------------------------------------------------------------- QRAdd_* */

/* Each variant orthogonalises v (= Delta f_{i-1}, modified in place) against
 * the k = m_i - 1 columns held, writes R[0:k-1][k] and returns rho. */

/* Algorithm 3 (Sec. 3.1): modified Gram-Schmidt, k + 1 reductions. */
static double add_mgs(ora_ctx *c, double *v, int k) {
  const int M = c->m;
  const int64_t n = c->n;
  for (int j = 0; j < k; ++j) {
    const double *qj = col(c->Q, n, j);
    double r = dot(qj, v, n);
    c->syncs_qr += 1;
    c->R[j * M + k] = r;
    ORA_PAR_FOR
    for (int64_t i = 0; i < n; ++i) v[i] -= r * qj[i];
  }
  double rho = nrm2(v, n);
  c->syncs_qr += 1;
  return rho;
}

/* Algorithm 4 (Sec. 3.2): inverse compact WY MGS.  The delayed row k-1 of T
 * and the projection coefficients come from one reduction; T is unit lower
 * (I + L) and is applied through forward substitution; then one reduction
 * for the norm. */
static double add_icwy(ora_ctx *c, double *v, int k) {
  const int M = c->m;
  const int64_t n = c->n;
  const double *qlast = col(c->Q, n, k - 1);
  for (int l = 0; l < k; ++l) c->T[(k - 1) * M + l] = dot(col(c->Q, n, l), qlast, n);
  for (int j = 0; j < k; ++j) c->R[j * M + k] = dot(col(c->Q, n, j), v, n);
  c->syncs_qr += 1;
  c->T[(k - 1) * M + (k - 1)] = 1.0;
  for (int j = 0; j < k; ++j) {
    double s = c->R[j * M + k];
    for (int l = 0; l < j; ++l) s -= c->T[j * M + l] * c->R[l * M + k];
    c->R[j * M + k] = s; /* unit diagonal */
  }
  for (int j = 0; j < k; ++j) {
    const double *qj = col(c->Q, n, j);
    double r = c->R[j * M + k];
    ORA_PAR_FOR
    for (int64_t i = 0; i < n; ++i) v[i] -= r * qj[i];
  }
  double rho = nrm2(v, n);
  c->syncs_qr += 1;
  return rho;
}

/* Algorithm 5 (Sec. 3.3): classical Gram-Schmidt with one full
 * reorthogonalisation; three reductions. */
static double add_cgs2(ora_ctx *c, double *v, int k) {
  const int M = c->m;
  const int64_t n = c->n;
  double s[256], z[256];
  for (int j = 0; j < k; ++j) s[j] = dot(col(c->Q, n, j), v, n);
  c->syncs_qr += 1;
  double *y = c->y;
  memcpy(y, v, sizeof(double) * (size_t)n);
  for (int j = 0; j < k; ++j) {
    const double *qj = col(c->Q, n, j);
    ORA_PAR_FOR
    for (int64_t i = 0; i < n; ++i) y[i] -= s[j] * qj[i];
  }
  for (int j = 0; j < k; ++j) z[j] = dot(col(c->Q, n, j), y, n);
  c->syncs_qr += 1;
  memcpy(v, y, sizeof(double) * (size_t)n);
  for (int j = 0; j < k; ++j) {
    const double *qj = col(c->Q, n, j);
    ORA_PAR_FOR
    for (int64_t i = 0; i < n; ++i) v[i] -= z[j] * qj[i];
  }
  for (int j = 0; j < k; ++j) c->R[j * M + k] = s[j] + z[j];
  double rho = nrm2(v, n);
  c->syncs_qr += 1;
  return rho;
}

/* Algorithm 6 (Sec. 3.4): CGS with delayed reorthogonalisation.  The
 * projection coefficients of v and, when m_i > 3, the reorthogonalisation
 * coefficients s of the previous column come from one reduction over the
 * current Q; the previous column is then corrected, R's previous column is
 * updated, and v is projected against the corrected Q; then one reduction
 * for the norm. */
static double add_dcgs2(ora_ctx *c, double *v, int k) {
  const int M = c->m;
  const int64_t n = c->n;
  const int mi = k + 1;
  double s[256];
  for (int j = 0; j < k; ++j) c->R[j * M + k] = dot(col(c->Q, n, j), v, n);
  int reorth = (mi > c->dcgs2_min_mi) && (k >= 2);
  double *qprev = col(c->Q, n, k - 1);
  if (reorth)
    for (int j = 0; j < k - 1; ++j) s[j] = dot(col(c->Q, n, j), qprev, n);
  c->syncs_qr += 1;
  if (reorth) {
    for (int j = 0; j < k - 1; ++j) {
      const double *qj = col(c->Q, n, j);
      ORA_PAR_FOR
      for (int64_t i = 0; i < n; ++i) qprev[i] -= s[j] * qj[i];
    }
    store_round_vec(c, qprev);
    double rkk = c->R[(k - 1) * M + (k - 1)];
    for (int j = 0; j < k - 1; ++j)
      c->R[j * M + (k - 1)] += c->dcgs2_scaled ? rkk * s[j] : s[j];
  }
  for (int j = 0; j < k; ++j) {
    const double *qj = col(c->Q, n, j);
    double r = c->R[j * M + k];
    ORA_PAR_FOR
    for (int64_t i = 0; i < n; ++i) v[i] -= r * qj[i];
  }
  double rho = nrm2(v, n);
  c->syncs_qr += 1;
  return rho;
}

/* Algorithm 2 (Sec. 2.1), QR part: delete the oldest column when the
 * history is full, then add v.  Returns ORA_OK or ORA_BREAKDOWN. */
int ora_qradd(ora_ctx *c, const double *vin) {
  const int64_t n = c->n;
  const int M = c->m;
  double *v = c->v;
  memcpy(v, vin, sizeof(double) * (size_t)n);
  double vnorm = nrm2(v, n);
  c->syncs_other += 1;
  if (!isfinite(vnorm)) {
    c->last_status = ORA_ENONFINITE;
    return ORA_ENONFINITE;
  }
  if (c->c == M) {
    qr_delete(c);
    if (c->orth == ORA_ICWY) icwy_refresh_T(c);
  }
  const int k = c->c;
  double rho;
  if (k == 0) {
    rho = vnorm;
    c->syncs_qr += 1; /* Algorithm 2, first column: one norm */
  } else {
    switch (c->orth) {
      case ORA_MGS: rho = add_mgs(c, v, k); break;
      case ORA_ICWY: rho = add_icwy(c, v, k); break;
      case ORA_CGS2: rho = add_cgs2(c, v, k); break;
      default: rho = add_dcgs2(c, v, k); break;
    }
  }
  if (!(rho > 0.0) || !isfinite(rho) || rho <= c->breakdown_tol * vnorm) {
    c->c = 0;
    c->last_status = ORA_BREAKDOWN;
    return ORA_BREAKDOWN;
  }
  c->R[k * M + k] = rho;
  double *qk = col(c->Q, n, k);
  ORA_PAR_FOR
  for (int64_t i = 0; i < n; ++i) qk[i] = v[i] / rho;
  store_round_vec(c, qk);
  if (c->orth == ORA_ICWY) {
    for (int l = 0; l < M; ++l) c->T[k * M + l] = 0.0;
    c->T[k * M + k] = 1.0;
  }
  c->c = k + 1;
  c->last_status = ORA_OK;
  return ORA_OK;
}

/* Algorithm 2, final step: solve R gamma = Q^T f by back-substitution. */
int ora_lsq(ora_ctx *c, const double *f, double *gamma) {
  const int k = c->c;
  const int M = c->m;
  double rhs[256];
  for (int j = 0; j < k; ++j) rhs[j] = dot(col(c->Q, c->n, j), f, c->n);
  if (k > 0) c->syncs_lsq += 1;
  for (int j = k - 1; j >= 0; --j) {
    double s = rhs[j];
    for (int l = j + 1; l < k; ++l) s -= c->R[j * M + l] * gamma[l];
    gamma[j] = s / c->R[j * M + j];
  }
  return k;
}

int ora_get_qr(const ora_ctx *c, double *Q, double *R, double *T, int *k) {
  *k = c->c;
  if (Q) memcpy(Q, c->Q, sizeof(double) * (size_t)c->n * c->c);
  if (R) memcpy(R, c->R, sizeof(double) * (size_t)c->m * c->m);
  if (T) memcpy(T, c->T, sizeof(double) * (size_t)c->m * c->m);
  return ORA_OK;
}

/* Seed Q, R directly (tests of QRDelete / QRAdd on prescribed factors). */
int ora_set_qr(ora_ctx *c, const double *Q, const double *R, const double *T, int k) {
  if (k < 0 || k > c->m) return ORA_EINVAL;
  c->c = k;
  memcpy(c->Q, Q, sizeof(double) * (size_t)c->n * k);
  memcpy(c->R, R, sizeof(double) * (size_t)c->m * c->m);
  if (T) memcpy(c->T, T, sizeof(double) * (size_t)c->m * c->m);
  return ORA_OK;
}

/* Exposed for the QRDelete unit tests. */
int ora_qrdelete(ora_ctx *c) {
  if (c->c < 1) return ORA_EINVAL;
  qr_delete(c);
  if (c->orth == ORA_ICWY) icwy_refresh_T(c);
  return ORA_OK;
}

/* ------------------------------------------------------------ AA step */

/* One iteration of Algorithm 1 given x_i and g_i = G(x_i).  Writes
 * x_{i+1} and returns ||f_i||_2 through fnorm.  Iteration 0 takes the plain
 * fixed-point step x_1 = G(x_0). */
int ora_step(ora_ctx *c, const double *x, const double *g, double *xnext, double *fnorm) {
  const int64_t n = c->n;
  const int M = c->m;
  double *f = c->f;
  ORA_PAR_FOR
  for (int64_t i = 0; i < n; ++i) f[i] = g[i] - x[i];
  double fn = nrm2(f, n);
  c->syncs_other += 1;
  if (fnorm) *fnorm = fn;
  if (!isfinite(fn)) return ORA_ENONFINITE;
  if (c->it == 0) {
    memcpy(c->f_prev, f, sizeof(double) * (size_t)n);
    memcpy(c->g_prev, g, sizeof(double) * (size_t)n);
    memcpy(xnext, g, sizeof(double) * (size_t)n);
    c->it = 1;
    return ORA_OK;
  }
  /* Delta f_{i-1} = f_i - f_{i-1}; Delta g_{i-1} = g_i - g_{i-1} */
  double *df = c->y; /* reuse as scratch before qradd copies it */
  double *dfcopy = (double *)malloc(sizeof(double) * (size_t)n);
  if (!dfcopy) return ORA_ENOMEM;
  ORA_PAR_FOR
  for (int64_t i = 0; i < n; ++i) dfcopy[i] = f[i] - c->f_prev[i];
  (void)df;
  int was_full = (c->c == M);
  int st = ora_qradd(c, dfcopy);
  free(dfcopy);
  if (st == ORA_ENONFINITE) return st;
  int ng; /* number of dG columns after this step */
  if (st == ORA_BREAKDOWN) {
    c->head = 0;
    ng = 0;
    memcpy(xnext, g, sizeof(double) * (size_t)n);
  } else {
    if (was_full) c->head = (c->head + 1) % M;
    ng = c->c;
    int slot = (c->head + ng - 1) % M;
    double *dg = col(c->dG, n, slot);
    ORA_PAR_FOR
    for (int64_t i = 0; i < n; ++i) dg[i] = g[i] - c->g_prev[i];
    store_round_vec(c, dg);
    double gamma[256];
    ora_lsq(c, f, gamma);
    /* x_{i+1} = g_i - dG_i gamma */
    memcpy(xnext, g, sizeof(double) * (size_t)n);
    for (int j = 0; j < ng; ++j) {
      const double *dgj = col(c->dG, n, (c->head + j) % M);
      ORA_PAR_FOR
      for (int64_t i = 0; i < n; ++i) xnext[i] -= gamma[j] * dgj[i];
    }
  }
  memcpy(c->f_prev, f, sizeof(double) * (size_t)n);
  memcpy(c->g_prev, g, sizeof(double) * (size_t)n);
  c->it += 1;
  return st;
}

/* ------------------------------------------------------- test problems */

/* 2D anisotropic 5-point Jacobi map: A has diagonal d = 2 + 2 eps, x
 * neighbours -1, y neighbours -eps, zero Dirichlet boundary; index
 * p = j*nx + i.  G(x) = x + D^{-1} (b - A x). */
void ora_g_jacobi2d(int64_t nx, int64_t ny, double eps, const double *b, const double *x,
                    double *gx) {
  const double d = 2.0 + 2.0 * eps;
  ORA_PAR_FOR
  for (int64_t j = 0; j < ny; ++j)
    for (int64_t i = 0; i < nx; ++i) {
      int64_t p = j * nx + i;
      double w = i > 0 ? x[p - 1] : 0.0;
      double e = i < nx - 1 ? x[p + 1] : 0.0;
      double s = j > 0 ? x[p - nx] : 0.0;
      double nn = j < ny - 1 ? x[p + nx] : 0.0;
      double ax = d * x[p] - (w + e) - eps * (s + nn);
      gx[p] = x[p] + (b[p] - ax) / d;
    }
}

/* 3D anisotropic 7-point weighted Jacobi: d = 2 (1 + ey + ez), neighbours
 * -1 (x), -ey (y), -ez (z); index p = (k*ny + j)*nx + i.
 * G(x) = x + omega D^{-1} (b - A x). */
void ora_g_jacobi3d(int64_t nx, int64_t ny, int64_t nz, double ey, double ez, double omega,
                    const double *b, const double *x, double *gx) {
  const double d = 2.0 * (1.0 + ey + ez);
  const int64_t sxy = nx * ny;
  ORA_PAR_FOR
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i) {
        int64_t p = (k * ny + j) * nx + i;
        double w = i > 0 ? x[p - 1] : 0.0;
        double e = i < nx - 1 ? x[p + 1] : 0.0;
        double s = j > 0 ? x[p - nx] : 0.0;
        double nn = j < ny - 1 ? x[p + nx] : 0.0;
        double dn = k > 0 ? x[p - sxy] : 0.0;
        double up = k < nz - 1 ? x[p + sxy] : 0.0;
        double ax = d * x[p] - (w + e) - ey * (s + nn) - ez * (dn + up);
        gx[p] = x[p] + omega * (b[p] - ax) / d;
      }
}

/* 2D Bratu nonlinear Jacobi on an s x s interior grid, h = 1/(s+1), zero
 * boundary: G(u)_p = (sum of the 4 neighbours + h^2 (lambda e^{u_p} + src_p)) / 4.
 * src may be NULL (pure Bratu, Sec. 5.2). */
void ora_g_bratu2d(int64_t s, double lambda, const double *src, const double *u, double *gu) {
  const double h = 1.0 / (double)(s + 1);
  const double h2 = h * h;
  ORA_PAR_FOR
  for (int64_t j = 0; j < s; ++j)
    for (int64_t i = 0; i < s; ++i) {
      int64_t p = j * s + i;
      double w = i > 0 ? u[p - 1] : 0.0;
      double e = i < s - 1 ? u[p + 1] : 0.0;
      double so = j > 0 ? u[p - s] : 0.0;
      double no = j < s - 1 ? u[p + s] : 0.0;
      double rhs = lambda * exp(u[p]) + (src ? src[p] : 0.0);
      gu[p] = ((w + e) + (so + no) + h2 * rhs) / 4.0;
    }
}

/* ------------------------------------------------------------ AA solve */

typedef void (*ora_gfn)(const double *x, double *gx, int64_t n, void *user);

typedef struct {
  int kind; /* 0 jacobi2d, 1 jacobi3d, 2 bratu2d, 3 callback */
  int64_t nx, ny, nz;
  double p0, p1, p2; /* eps | ey, ez, omega | lambda */
  const double *b;   /* rhs or source (may be NULL for bratu) */
  ora_gfn fn;
  void *user;
} ora_problem;

static void eval_g(const ora_problem *P, const double *x, double *gx, int64_t n) {
  switch (P->kind) {
    case 0: ora_g_jacobi2d(P->nx, P->ny, P->p0, P->b, x, gx); break;
    case 1: ora_g_jacobi3d(P->nx, P->ny, P->nz, P->p0, P->p1, P->p2, P->b, x, gx); break;
    case 2: ora_g_bratu2d(P->nx, P->p0, P->b, x, gx); break;
    default: P->fn(x, gx, n, P->user); break;
  }
}

/* Algorithm 1.  Stop rule (stop_kind 0): ||G(x_i) - x_i||_2 / scale < tol,
 * tested on f_i before the least-squares solve; x_i is returned and the
 * iteration count is i.  stop_kind 1 is the paper's ||x_{i+1} - x_i|| < tol
 * (2-norm), returning x_{i+1} with count i + 1.  Records ||f_i|| in
 * resid[0..] and the first nrec iterates x_1.. in rec (n doubles each). */
int ora_solve(ora_ctx *c, const ora_problem *P, double *x, int max_iters, double tol,
              double scale, int stop_kind, int nrec, double *rec, double *resid, int *iters) {
  const int64_t n = c->n;
  double *g = (double *)malloc(sizeof(double) * (size_t)n);
  double *xn = (double *)malloc(sizeof(double) * (size_t)n);
  if (!g || !xn) {
    free(g); free(xn);
    return ORA_ENOMEM;
  }
  ora_reset(c);
  int status = ORA_NOTCONVERGED;
  int i;
  for (i = 0;; ++i) {
    eval_g(P, x, g, n);
    double fn;
    int st = ora_step(c, x, g, xn, &fn);
    if (resid) resid[i] = fn;
    if (st == ORA_ENONFINITE) { status = st; break; }
    if (stop_kind == 0 && fn / scale < tol) { status = ORA_OK; break; }
    if (i == max_iters) break;
    if (stop_kind == 1) {
      double d = 0.0;
      for (int64_t p = 0; p < n; ++p) d += (xn[p] - x[p]) * (xn[p] - x[p]);
      memcpy(x, xn, sizeof(double) * (size_t)n);
      if (i < nrec && rec) memcpy(rec + (size_t)i * n, x, sizeof(double) * (size_t)n);
      if (sqrt(d) < tol) { status = ORA_OK; ++i; break; }
    } else {
      memcpy(x, xn, sizeof(double) * (size_t)n);
      if (i < nrec && rec) memcpy(rec + (size_t)i * n, x, sizeof(double) * (size_t)n);
    }
  }
  if (iters) *iters = i;
  free(g);
  free(xn);
  return status;
}
