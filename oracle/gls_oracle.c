/*
 * FP64 CPU oracle for the per-SNP generalized least-squares (GLS) sequence.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference against
 * which the CUDA path is checked.  Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or helper with the CUDA library, and it includes nothing
 * from it.
 *
 * What it computes (Beyer & Bientinesi, "Streaming Data from HDD to GPUs for
 * Sustained Peak Performance"):
 *
 *   Eq. 1   r_i = (X_i^T M^-1 X_i)^-1 X_i^T M^-1 y,        i = 1..m
 *           with X_i = (X_L | X_R_i)  (Sec. 1.3): X_L the n x (p-1) fixed
 *           covariates, X_R_i the i-th SNP column.  The SNP coefficient is the
 *           last entry of r_i.
 *   Eq. 2   with L L^T = M:  X~_i = L^-1 X_i,  y~ = L^-1 y,
 *           r_i = (X~_i^T X~_i)^-1 X~_i^T y~.
 *   Listing 1 (Sec. 2.1): X~_L, y~, r_T = X~_L^T y~ and S_TL = X~_L^T X~_L are
 *           computed once; per SNP: x~_i = L^-1 x_i (trsv), S_BL = x~_i^T X~_L,
 *           S_BR = x~_i^T x~_i, r_B = x~_i^T y~, then the p x p SPD solve (posv).
 *   Sec. 2.2: several SNP columns are solved together (trsv -> trsm); here a
 *           group of columns shares one sweep over L, nothing more.
 *
 * M = sigma2 (h Phi + (1 - h) I) is the variance-component form of M that the
 * paper leaves open (it says only that M models the relations among the
 * samples, Sec. 1.3).
 *
 * Readings added to the paper (none is stated there):
 *   - standard errors: se_j = sqrt((S^-1)_jj) with S = X_i^T M^-1 X_i (M known,
 *     sigma2 included); Wald chi2 = r_{p-1}^2 / (S^-1)_{p-1,p-1};
 *   - a SNP whose design is numerically collinear, i.e. whose last Cholesky
 *     pivot of S satisfies  d^2 <= ORACLE_SINGULAR_TAU * S_{p-1,p-1}  (or any
 *     pivot of the covariate block fails the same test), gets status 1 and
 *     NaN in r, se and chi2; the block is never aborted.
 *
 * Column-major storage throughout: element (i, j) of an n-row matrix is at
 * [i + j * n].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_SINGULAR_TAU 1e-7
#define ORACLE_GROUP 16 /* SNP columns per sweep over L (Sec. 2.2 trsv -> trsm) */

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_set_num_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

/* M = sigma2 * (h * Phi + (1 - h) * I).  Phi and M are n x n. */
void oracle_form_m(int64_t n, const double *phi, double h, double sigma2, double *M) {
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) {
      double v = h * phi[i + j * n];
      if (i == j) v += 1.0 - h;
      M[i + j * n] = sigma2 * v;
    }
}

/* Textbook right-looking Cholesky, L L^T = A, lower triangle in place
 * (Sec. 2.1: "potrf M").  The strict upper triangle is set to zero.
 * Returns -1 on success, else the index of the first pivot that is not
 * strictly positive. */
int64_t oracle_potrf(int64_t n, double *A) {
  for (int64_t j = 0; j < n; ++j) {
    double d = A[j + j * n];
    if (!(d > 0.0)) return j;
    d = sqrt(d);
    A[j + j * n] = d;
    for (int64_t i = j + 1; i < n; ++i) A[i + j * n] /= d;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = j + 1; k < n; ++k) {
      const double lkj = A[k + j * n];
      double *colk = A + k * n;
      const double *colj = A + j * n;
      for (int64_t i = k; i < n; ++i) colk[i] -= colj[i] * lkj;
    }
  }
  for (int64_t j = 1; j < n; ++j)
    for (int64_t i = 0; i < j; ++i) A[i + j * n] = 0.0;
  return -1;
}

/* Forward substitution L x = b for `ncols` right-hand sides at once.
 * X is n x ncols with leading dimension ldx and is overwritten by L^-1 X.
 * Column-oriented sweep: L is read once for the whole group. */
static void forward_subst(int64_t n, const double *L, int64_t ncols, double *X, int64_t ldx) {
  for (int64_t j = 0; j < n; ++j) {
    const double ljj = L[j + j * n];
    for (int64_t c = 0; c < ncols; ++c) X[j + c * ldx] /= ljj;
    const double *colj = L + j * n;
    for (int64_t c = 0; c < ncols; ++c) {
      const double xj = X[j + c * ldx];
      double *xc = X + c * ldx;
      for (int64_t i = j + 1; i < n; ++i) xc[i] -= colj[i] * xj;
    }
  }
}

void oracle_trsm_lower(int64_t n, const double *L, int64_t ncols, double *X) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t c0 = 0; c0 < ncols; c0 += ORACLE_GROUP) {
    int64_t g = ncols - c0 < ORACLE_GROUP ? ncols - c0 : ORACLE_GROUP;
    forward_subst(n, L, g, X + c0 * n, n);
  }
}

static double dot(int64_t n, const double *a, const double *b) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* posv on a p x p SPD matrix S (column-major, overwritten by its Cholesky
 * factor).  Solves S r = rhs and forms diag(S^-1).  Returns 0, or 1 when a
 * pivot fails the collinearity test. */
static int posv_small(int p, double *S, const double *rhs, double *r, double *diag_inv) {
  double diag0[64];
  for (int j = 0; j < p; ++j) diag0[j] = S[j + j * p];
  for (int j = 0; j < p; ++j) {
    double d = S[j + j * p];
    for (int k = 0; k < j; ++k) d -= S[j + k * p] * S[j + k * p];
    if (!(d > ORACLE_SINGULAR_TAU * diag0[j])) return 1;
    d = sqrt(d);
    S[j + j * p] = d;
    for (int i = j + 1; i < p; ++i) {
      double v = S[i + j * p];
      for (int k = 0; k < j; ++k) v -= S[i + k * p] * S[j + k * p];
      S[i + j * p] = v / d;
    }
  }
  /* forward then backward substitution */
  double z[64];
  for (int i = 0; i < p; ++i) {
    double v = rhs[i];
    for (int k = 0; k < i; ++k) v -= S[i + k * p] * z[k];
    z[i] = v / S[i + i * p];
  }
  for (int i = p - 1; i >= 0; --i) {
    double v = z[i];
    for (int k = i + 1; k < p; ++k) v -= S[k + i * p] * r[k];
    r[i] = v / S[i + i * p];
  }
  /* diag(S^-1): solve S w = e_j for every j and keep w_j */
  for (int j = 0; j < p; ++j) {
    double w[64];
    for (int i = 0; i < p; ++i) {
      double v = (i == j) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) v -= S[i + k * p] * w[k];
      w[i] = v / S[i + i * p];
    }
    for (int i = p - 1; i >= 0; --i) {
      double v = w[i];
      for (int k = i + 1; k < p; ++k) v -= S[k + i * p] * w[k];
      w[i] = v / S[i + i * p];
    }
    diag_inv[j] = w[j];
  }
  return 0;
}

/* The GLS sequence (Eq. 1 via Eq. 2, loop structure of Listing 1).
 *
 *   L   n x n lower Cholesky factor of M (upper triangle ignored)
 *   XL  n x (p-1) fixed covariates,  y  n,  XR  n x m SNP columns (float64)
 *   r, se  p x m outputs; chi2 m (may be NULL); status m (may be NULL)
 *
 * Returns 0, or -1 on bad arguments or when S_TL itself is singular. */
int oracle_gls(int64_t n, int p, const double *L, const double *XL, const double *y, int64_t m,
               const double *XR, double *r, double *se, double *chi2, int *status) {
  if (n < 1 || p < 1 || p > 64 || m < 0) return -1;
  const int q = p - 1;
  /* Listing 1, loop-invariant part: X~_L, y~, r_T, S_TL */
  double *XLt = (double *)malloc(sizeof(double) * (size_t)n * (size_t)(q + 1));
  if (!XLt) return -1;
  if (q) memcpy(XLt, XL, sizeof(double) * (size_t)n * (size_t)q);
  memcpy(XLt + (size_t)q * n, y, sizeof(double) * (size_t)n);
  forward_subst(n, L, q + 1, XLt, n);
  const double *yt = XLt + (size_t)q * n;
  double STL[64 * 64], rT[64];
  for (int a = 0; a < q; ++a) {
    rT[a] = dot(n, XLt + (size_t)a * n, yt);
    for (int b = 0; b < q; ++b) STL[a + b * 64] = dot(n, XLt + (size_t)a * n, XLt + (size_t)b * n);
  }

  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t c0 = 0; c0 < m; c0 += ORACLE_GROUP) {
    const int64_t g = m - c0 < ORACLE_GROUP ? m - c0 : ORACLE_GROUP;
    double *Xt = (double *)malloc(sizeof(double) * (size_t)n * (size_t)g);
    if (!Xt) {
#pragma omp atomic write
      bad = 1;
      continue;
    }
    memcpy(Xt, XR + (size_t)c0 * n, sizeof(double) * (size_t)n * (size_t)g);
    forward_subst(n, L, g, Xt, n); /* x~_i = L^-1 x_i (trsv, grouped) */
    for (int64_t c = 0; c < g; ++c) {
      const int64_t i = c0 + c;
      const double *xt = Xt + (size_t)c * n;
      double S[64 * 64], rhs[64], ri[64], dinv[64];
      for (int a = 0; a < q; ++a) {
        for (int b = 0; b < q; ++b) S[a + b * p] = STL[a + b * 64];
        const double sbl = dot(n, xt, XLt + (size_t)a * n); /* S_BL */
        S[q + a * p] = sbl;
        S[a + q * p] = sbl;
        rhs[a] = rT[a];
      }
      S[q + q * p] = dot(n, xt, xt); /* S_BR */
      rhs[q] = dot(n, xt, yt);       /* r_B */
      int st = posv_small(p, S, rhs, ri, dinv);
      for (int j = 0; j < p; ++j) {
        r[j + i * p] = st ? NAN : ri[j];
        se[j + i * p] = st ? NAN : sqrt(dinv[j]);
      }
      if (chi2) chi2[i] = st ? NAN : ri[q] * ri[q] / dinv[q];
      if (status) status[i] = st;
    }
    free(Xt);
  }
  free(XLt);
  return bad ? -1 : 0;
}
