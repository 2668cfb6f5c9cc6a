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

/* ------------------------------------------------------------------------
 * Gradients (the differentiation form; not in the paper).
 *
 * Per SNP, with W = M^-1, S = X^T W X, b = S^-1 X^T W y, v = S^-1 e_{p-1},
 * s = v_{p-1}, Wald chi2 = b_{p-1}^2 / s, a = X v, e = y - X b:
 *   d chi2 / dy = (2 b_{p-1} / s) W a
 *   d chi2 / dh = -(2 b_{p-1} / s) (W a)^T D (W e) - (b_{p-1}^2 / s^2) (W a)^T D (W a),
 *   D = dM/dh = sigma2 (Phi - I).
 * W z is computed as a forward then a backward substitution with L.
 * ------------------------------------------------------------------------ */

/* In place: x <- M^-1 x = L^-T (L^-1 x). */
static void solve_m(int64_t n, const double *L, double *x) {
  for (int64_t j = 0; j < n; ++j) { /* forward: L z = x */
    x[j] /= L[j + j * n];
    const double xj = x[j];
    for (int64_t i = j + 1; i < n; ++i) x[i] -= L[i + j * n] * xj;
  }
  for (int64_t i = n - 1; i >= 0; --i) { /* backward: L^T w = z */
    double v = x[i];
    for (int64_t k = i + 1; k < n; ++k) v -= L[k + i * n] * x[k];
    x[i] = v / L[i + i * n];
  }
}

/* D z = sigma2 (Phi z - z). */
static void apply_d(int64_t n, const double *phi, double sigma2, const double *z, double *out) {
  for (int64_t i = 0; i < n; ++i) out[i] = -z[i];
  for (int64_t j = 0; j < n; ++j) {
    const double zj = z[j];
    const double *col = phi + j * n;
    for (int64_t i = 0; i < n; ++i) out[i] += col[i] * zj;
  }
  for (int64_t i = 0; i < n; ++i) out[i] *= sigma2;
}

/* chi2[m], dchi2_dh[m] per SNP and dy[n] = sum over SNPs of d chi2 / dy.
 * Returns 0, or -1 on bad arguments.  Singular SNPs contribute nothing and
 * get NaN. */
int oracle_gls_grad(int64_t n, int p, const double *L, const double *phi, double h, double sigma2,
                    const double *XL, const double *y, int64_t m, const double *XR, double *chi2,
                    double *dchi2_dh, double *dy) {
  if (n < 1 || p < 1 || p > 64 || m < 0) return -1;
  const int q = p - 1;
  for (int64_t i = 0; i < n; ++i) dy[i] = 0.0;
  int bad = 0;
#pragma omp parallel
  {
    double *X = (double *)malloc(sizeof(double) * (size_t)n * (size_t)(p + 1)); /* [X_i | y], then solved */
    double *a = (double *)malloc(sizeof(double) * (size_t)n);
    double *e = (double *)malloc(sizeof(double) * (size_t)n);
    double *Da = (double *)malloc(sizeof(double) * (size_t)n);
    double *De = (double *)malloc(sizeof(double) * (size_t)n);
    double *dy_local = (double *)calloc((size_t)n, sizeof(double));
    if (!X || !a || !e || !Da || !De || !dy_local) {
#pragma omp atomic write
      bad = 1;
    } else {
#pragma omp for schedule(dynamic, 1)
      for (int64_t i = 0; i < m; ++i) {
        if (q) memcpy(X, XL, sizeof(double) * (size_t)n * q);
        memcpy(X + (size_t)q * n, XR + (size_t)i * n, sizeof(double) * (size_t)n);
        memcpy(X + (size_t)p * n, y, sizeof(double) * (size_t)n);
        forward_subst(n, L, p + 1, X, n); /* X~ = L^-1 [X_i | y] */
        const double *yt = X + (size_t)p * n;
        double S[64 * 64], r[64], bb[64], v[64], dinv[64], ev[64];
        for (int c = 0; c < p; ++c) {
          r[c] = dot(n, X + (size_t)c * n, yt);
          for (int d = 0; d < p; ++d) S[c + d * p] = dot(n, X + (size_t)c * n, X + (size_t)d * n);
        }
        double Sc[64 * 64];
        memcpy(Sc, S, sizeof(double) * p * p);
        int st = posv_small(p, Sc, r, bb, dinv);
        if (st) {
          chi2[i] = NAN;
          dchi2_dh[i] = NAN;
          continue;
        }
        for (int c = 0; c < p; ++c) ev[c] = (c == q) ? 1.0 : 0.0;
        memcpy(Sc, S, sizeof(double) * p * p);
        posv_small(p, Sc, ev, v, dinv); /* v = S^-1 e_{p-1} */
        const double s = v[q], bp = bb[q];
        chi2[i] = bp * bp / s;
        /* a = X v, e = y - X b with the original (unsolved) columns */
        for (int64_t t = 0; t < n; ++t) {
          double av = 0.0, xb = 0.0;
          for (int c = 0; c < q; ++c) {
            av += XL[t + (size_t)c * n] * v[c];
            xb += XL[t + (size_t)c * n] * bb[c];
          }
          av += XR[t + (size_t)i * n] * v[q];
          xb += XR[t + (size_t)i * n] * bb[q];
          a[t] = av;
          e[t] = y[t] - xb;
        }
        solve_m(n, L, a); /* W a */
        solve_m(n, L, e); /* W e */
        apply_d(n, phi, sigma2, a, Da);
        apply_d(n, phi, sigma2, e, De);
        dchi2_dh[i] = -(2.0 * bp / s) * dot(n, a, De) - (bp * bp / (s * s)) * dot(n, a, Da);
        const double cy = 2.0 * bp / s;
        for (int64_t t = 0; t < n; ++t) dy_local[t] += cy * a[t];
      }
#pragma omp critical
      for (int64_t t = 0; t < n; ++t) dy[t] += dy_local[t];
    }
    free(X);
    free(a);
    free(e);
    free(Da);
    free(De);
    free(dy_local);
  }
  return bad ? -1 : 0;
}

/* ------------------------------------------------------------------------
 * REML of the null model y ~ N(X_L beta, sigma2 V), V = h Phi + (1 - h) I,
 * sigma2 profiled out (q = p - 1 covariates):
 *   l(h) = -1/2 [ (n - q) log s2 + log|V| + log|X_L^T V^-1 X_L| ],
 *   s2 = y^T P y / (n - q),  P = V^-1 - V^-1 X_L (X_L^T V^-1 X_L)^-1 X_L^T V^-1,
 *   dl/dh = -1/2 [ tr(P (Phi - I)) - y^T P (Phi - I) P y / s2 ].
 * out[0] = l(h), out[1] = dl/dh (only when want_grad), out[2] = s2.
 * P is formed explicitly (dense, n^3): a plain evaluation, not a fast one.
 * Returns 0, or the 1-based index of a failing pivot (V or X_L^T V^-1 X_L).
 * ------------------------------------------------------------------------ */
int64_t oracle_reml(int64_t n, int q, const double *phi, const double *XL, const double *y, double h,
                    int want_grad, double *out) {
  double *Lv = (double *)malloc(sizeof(double) * (size_t)n * n);
  double *Xt = (double *)malloc(sizeof(double) * (size_t)n * (q + 1));
  if (!Lv || !Xt) { free(Lv); free(Xt); return -1; }
  oracle_form_m(n, phi, h, 1.0, Lv);
  int64_t bad = oracle_potrf(n, Lv);
  if (bad >= 0) { free(Lv); free(Xt); return bad + 1; }
  double logdetV = 0.0;
  for (int64_t i = 0; i < n; ++i) logdetV += 2.0 * log(Lv[i + i * n]);
  if (q) memcpy(Xt, XL, sizeof(double) * (size_t)n * q);
  memcpy(Xt + (size_t)q * n, y, sizeof(double) * (size_t)n);
  forward_subst(n, Lv, q + 1, Xt, n);
  double A[64 * 64], Ac[64 * 64], rhs[64], beta[64], dinv[64];
  for (int a = 0; a < q; ++a) {
    rhs[a] = dot(n, Xt + (size_t)a * n, Xt + (size_t)q * n);
    for (int b = 0; b < q; ++b) A[a + b * q] = dot(n, Xt + (size_t)a * n, Xt + (size_t)b * n);
  }
  double logdetA = 0.0;
  if (q) {
    memcpy(Ac, A, sizeof(double) * q * q);
    if (posv_small(q, Ac, rhs, beta, dinv)) { free(Lv); free(Xt); return n + 1; }
    for (int a = 0; a < q; ++a) logdetA += 2.0 * log(Ac[a + a * q]);
  }
  /* y^T P y = || y~ - X~_L beta ||^2 */
  double yPy = 0.0;
  for (int64_t t = 0; t < n; ++t) {
    double r = Xt[t + (size_t)q * n];
    for (int a = 0; a < q; ++a) r -= Xt[t + (size_t)a * n] * beta[a];
    yPy += r * r;
  }
  const double s2 = yPy / (double)(n - q);
  out[0] = -0.5 * ((double)(n - q) * log(s2) + logdetV + logdetA);
  out[2] = s2;
  if (want_grad) {
    /* explicit P: Vinv = L^-T L^-1, then P = Vinv - (Vinv X_L) A^-1 (Vinv X_L)^T */
    double *Vinv = (double *)malloc(sizeof(double) * (size_t)n * n);
    double *VX = (double *)malloc(sizeof(double) * (size_t)n * (q + 1));
    double *Py = (double *)malloc(sizeof(double) * (size_t)n);
    double *tmp = (double *)malloc(sizeof(double) * (size_t)n);
    if (!Vinv || !VX || !Py || !tmp) { free(Lv); free(Xt); free(Vinv); free(VX); free(Py); free(tmp); return -1; }
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t j = 0; j < n; ++j) {
      double *col = Vinv + (size_t)j * n;
      for (int64_t i = 0; i < n; ++i) col[i] = (i == j) ? 1.0 : 0.0;
      solve_m(n, Lv, col);
    }
    for (int a = 0; a < q; ++a) {
      memcpy(VX + (size_t)a * n, XL + (size_t)a * n, sizeof(double) * (size_t)n);
      solve_m(n, Lv, VX + (size_t)a * n);
    }
    double Ainv[64 * 64];
    for (int c = 0; c < q; ++c) {
      double ec[64], col[64];
      for (int a = 0; a < q; ++a) ec[a] = (a == c) ? 1.0 : 0.0;
      memcpy(Ac, A, sizeof(double) * q * q);
      posv_small(q, Ac, ec, col, dinv);
      for (int a = 0; a < q; ++a) Ainv[a + c * q] = col[a];
    }
    /* P in place of Vinv */
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j)
      for (int64_t i = 0; i < n; ++i) {
        double v = 0.0;
        for (int a = 0; a < q; ++a)
          for (int b = 0; b < q; ++b) v += VX[i + (size_t)a * n] * Ainv[a + b * q] * VX[j + (size_t)b * n];
        Vinv[i + (size_t)j * n] -= v;
      }
    /* tr(P (Phi - I)) and y^T P (Phi - I) P y */
    double tr = 0.0;
#pragma omp parallel for reduction(+ : tr) schedule(static)
    for (int64_t j = 0; j < n; ++j)
      for (int64_t i = 0; i < n; ++i) tr += Vinv[i + (size_t)j * n] * (phi[j + (size_t)i * n] - (i == j ? 1.0 : 0.0));
    for (int64_t i = 0; i < n; ++i) {
      double v = 0.0;
      for (int64_t j = 0; j < n; ++j) v += Vinv[i + (size_t)j * n] * y[j];
      Py[i] = v;
    }
    apply_d(n, phi, 1.0, Py, tmp);
    const double quad = dot(n, Py, tmp);
    out[1] = -0.5 * (tr - quad / s2);
    free(Vinv);
    free(VX);
    free(Py);
    free(tmp);
  }
  free(Lv);
  free(Xt);
  return 0;
}
