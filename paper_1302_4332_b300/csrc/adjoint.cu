// a11, the differentiation form (not in the paper): d(sum of per-SNP Wald
// chi2)/dh and /dy, FP64.
//
// Per SNP, with W = M^-1, S = X^T W X, b = S^-1 X^T W y, v = S^-1 e_p
// (p = last index), s = v_p, chi2 = b_p^2 / s, a = X v, e = y - X b:
//   d chi2 / dy = (2 b_p / s) W a,
//   d chi2 / dh = -(2 b_p / s) (W a)^T D (W e) - (b_p^2 / s^2) (W a)^T D (W a),
//   D = dM/dh = sigma2 (Phi - I) = (M - sigma2 I) / h   (h > 0).
// With W M W = W and a^T W e = v^T (X^T W y - S b) = 0:
//   (W a)^T D (W e) = -(sigma2 / h) (W a)^T (W e),
//   (W a)^T D (W a) = (s - sigma2 ||W a||^2) / h,
// so d chi2/dh = (1/h) [ (2 sigma2 b_p / s) ea - b_p^2 / s + (sigma2 b_p^2 / s^2) aa ]
// with ea = (W e)^T (W a) and aa = ||W a||^2.  Both need X^ = M^-1 X =
// L^-T X~ (the transpose solve): with T = X^T M^-2 X = X^^T X^,
//   aa = v^T T v,   ea = y^^T X^ v - b^T T v   (y^ = M^-1 y).
// T and y^^T X^ split into a loop-invariant part (X^_L, y^) and per-SNP
// sums of x^ against [X^_L | y^] and itself, exactly like the forward sums.
// The y-gradient sums over SNPs: sum_i c_i W a_i = X^_L (sum_i c_i v_T,i)
// + sum_i c_i v_p,i x^_i,  c_i = 2 b_p / s.
#include "gwas_internal.cuh"

namespace gwas {

// One warp per SNP: forward sums of x~ against W = [X~_L | y~] and transpose
// sums of x^ against What = [X^_L | y^], then the p x p adjoint.
template <int QM>
__global__ void __launch_bounds__(256) adjoint_snp_kernel(const double* __restrict__ Xt, const double* __restrict__ Xh,
                                                          int64_t ldt, int rows, const double* __restrict__ W,
                                                          const double* __restrict__ Wh, int64_t ldw,
                                                          const SolveConsts* __restrict__ sc,
                                                          const double* __restrict__ GH, int q, int ncols, double h,
                                                          double sigma2, double* __restrict__ chi2,
                                                          double* __restrict__ dh, double* __restrict__ wv) {
  const int lane = threadIdx.x & 31;
  const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (col >= ncols) return;
  const double* xt = Xt + (int64_t)col * ldt;
  const double* xh = Xh + (int64_t)col * ldt;
  double af[QM + 2], ah[QM + 2];
#pragma unroll
  for (int a = 0; a < QM + 2; ++a) af[a] = ah[a] = 0.0;
  for (int r = lane; r < rows; r += 32) {
    const double u = __ldcs(xt + r), w = __ldcs(xh + r);
#pragma unroll
    for (int a = 0; a <= QM; ++a)
      if (a <= q) {
        af[a] = fma(u, W[r + a * ldw], af[a]);
        ah[a] = fma(w, Wh[r + a * ldw], ah[a]);
      }
    af[QM + 1] = fma(u, u, af[QM + 1]);
    ah[QM + 1] = fma(w, w, ah[QM + 1]);
  }
#pragma unroll
  for (int a = 0; a < QM + 2; ++a)
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      af[a] += __shfl_xor_sync(0xffffffffu, af[a], o);
      ah[a] += __shfl_xor_sync(0xffffffffu, ah[a], o);
    }
  if (lane != 0) return;

  const int p = q + 1, nc = q + 1;
  // forward: l = C^-1 S_BL, d^2, b, g = C^-T l (as in the block solve)
  double l[QM > 0 ? QM : 1], g[QM > 0 ? QM : 1];
  double ll = 0.0, lz = 0.0;
  for (int i = 0; i < q; ++i) {
    double v = 0.0;
    for (int t = 0; t <= i; ++t) v = fma(sc->Cinv[i + t * QMAX], af[t], v);
    l[i] = v;
    ll = fma(v, v, ll);
    lz = fma(v, sc->zT[i], lz);
  }
  const double sbr = af[QM + 1], rb = af[q];
  const double d2 = sbr - ll;
  double* w_out = wv + (int64_t)col * p;
  if (!(d2 > SINGULAR_TAU * sbr)) {
    chi2[col] = __longlong_as_double(0x7ff8000000000000LL);
    dh[col] = 0.0;  // a collinear SNP adds nothing to the sums
    for (int j = 0; j < p; ++j) w_out[j] = 0.0;
    return;
  }
  const double bp = (rb - lz) / d2;
  double bT[QM > 0 ? QM : 1];
  for (int j = 0; j < q; ++j) {
    double v = 0.0;
    for (int i = j; i < q; ++i) v = fma(sc->Cinv[i + j * QMAX], l[i], v);
    g[j] = v;
    bT[j] = sc->b0[j] - bp * v;
  }
  // v = S^-1 e_p:  v_p = 1/d^2, v_T = -g/d^2;  s = v_p
  const double vp = 1.0 / d2, s = vp;
  double vT[QM > 0 ? QM : 1];
  for (int j = 0; j < q; ++j) vT[j] = -g[j] * vp;
  // T v with T = [[T_LL, t], [t^T, tau]],  t = x^ . X^_L,  tau = x^ . x^
  double TvT[QM > 0 ? QM : 1];
  double Tvp = ah[QM + 1] * vp;
  for (int i = 0; i < q; ++i) {
    double v = ah[i] * vp;
    for (int j = 0; j < q; ++j) v = fma(GH[i + j * nc], vT[j], v);
    TvT[i] = v;
    Tvp = fma(ah[i], vT[i], Tvp);
  }
  double aa = vp * Tvp, ea = ah[q] * vp - bp * Tvp;
  for (int i = 0; i < q; ++i) {
    aa = fma(vT[i], TvT[i], aa);
    ea = fma(GH[q + i * nc], vT[i], ea);  // y^ . X^_L
    ea = fma(-bT[i], TvT[i], ea);
  }
  chi2[col] = bp * bp / s;
  dh[col] = ((2.0 * sigma2 * bp / s) * ea - bp * bp / s + (sigma2 * bp * bp / (s * s)) * aa) / h;
  const double c = 2.0 * bp / s;
  for (int j = 0; j < q; ++j) w_out[j] = c * vT[j];
  w_out[q] = c * vp;
}

// One block: dh_sum += sum_i dh_i and uT[a] = sum_i w_i[a] (a < q), in a fixed order.
__global__ void adjoint_sum_kernel(const double* __restrict__ dh, const double* __restrict__ wv, int q, int ncols,
                                   double* __restrict__ dh_accum, double* __restrict__ uT) {
  __shared__ double red[QMAX + 1][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;  // warp a < q: uT[a]; warp q: dh
  if (warp > q) return;
  double s = 0.0;
  for (int i = lane; i < ncols; i += 32) s += (warp == q) ? dh[i] : wv[(int64_t)i * (q + 1) + warp];
  red[warp][lane] = s;
  __syncwarp();
  if (lane == 0) {
    double t = 0.0;
    for (int l = 0; l < 32; ++l) t += red[warp][l];
    if (warp == q)
      *dh_accum += t;
    else
      uT[warp] = t;
  }
}

// dy[r] += sum_a uT[a] X^_L[r, a] + sum_i w_p,i x^_i[r]   (r < n)
__global__ void adjoint_dy_kernel(const double* __restrict__ Xh, int64_t ldt, const double* __restrict__ Wh,
                                  int64_t ldw, const double* __restrict__ wv, const double* __restrict__ uT, int q,
                                  int n, int ncols, double* __restrict__ dy) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double s = 0.0;
  for (int a = 0; a < q; ++a) s = fma(uT[a], Wh[r + a * ldw], s);
  for (int i = 0; i < ncols; ++i) s = fma(wv[(int64_t)i * (q + 1) + q], Xh[r + (int64_t)i * ldt], s);
  dy[r] += s;
}

cudaError_t launch_adjoint(const double* Xt, const double* Xh, int64_t ldt, int rows, int n, const double* W,
                           const double* Wh, int64_t ldw, const SolveConsts* sc, const double* GH, int q,
                           int ncols, double h, double sigma2, double* chi2, double* dh, double* wv, double* uT,
                           double* dh_accum, double* dy_accum, cudaStream_t s) {
  if (ncols <= 0) return cudaSuccess;
  const int grid = (ncols + 7) / 8;
  if (q <= 3)
    adjoint_snp_kernel<3><<<grid, 256, 0, s>>>(Xt, Xh, ldt, rows, W, Wh, ldw, sc, GH, q, ncols, h, sigma2, chi2, dh, wv);
  else if (q <= 7)
    adjoint_snp_kernel<7><<<grid, 256, 0, s>>>(Xt, Xh, ldt, rows, W, Wh, ldw, sc, GH, q, ncols, h, sigma2, chi2, dh, wv);
  else
    adjoint_snp_kernel<QMAX><<<grid, 256, 0, s>>>(Xt, Xh, ldt, rows, W, Wh, ldw, sc, GH, q, ncols, h, sigma2, chi2, dh,
                                                  wv);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  adjoint_sum_kernel<<<1, 32 * (q + 1), 0, s>>>(dh, wv, q, ncols, dh_accum, uT);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  adjoint_dy_kernel<<<(n + 255) / 256, 256, 0, s>>>(Xh, ldt, Wh, ldw, wv, uT, q, n, ncols, dy_accum);
  return cudaGetLastError();
}

// ----------------------------------------------------------- REML helpers
// out[0] = sum log(L_ii) over i < n;  out[1] = sum of squares of X (rows < n, cols < ncols)
__global__ void log_diag_kernel(const double* __restrict__ L, int64_t ld, int n, double* __restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += log(L[i + i * ld]);
  red[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < blockDim.x; ++i) t += red[i];
    *out = t;
  }
}

// out[c] = sum over rows < n of X[r, c]^2 (one block per column)
__global__ void col_sumsq_kernel(const double* __restrict__ X, int64_t ld, int n, double* __restrict__ out) {
  __shared__ double red[256];
  const double* x = X + (int64_t)blockIdx.x * ld;
  double s = 0.0;
  for (int r = threadIdx.x; r < n; r += blockDim.x) s = fma(x[r], x[r], s);
  red[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < blockDim.x; ++i) t += red[i];
    out[blockIdx.x] = t;
  }
}

// n x ncols columns c0 .. c0+ncols-1 of the identity (column-major, ld n)
__global__ void identity_cols_kernel(double* __restrict__ E, int n, int c0, int ncols) {
  const int64_t total = (int64_t)n * ncols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % n), c = (int)(e / n);
    E[e] = (r == c0 + c) ? 1.0 : 0.0;
  }
}

// residual r~ = y~ - X~_L beta (beta = S_TL^-1 r_T), rows < n_pad, into R
__global__ void null_residual_kernel(const double* __restrict__ W, int64_t ldw, int rows, int q,
                                     const SolveConsts* __restrict__ sc, double* __restrict__ R) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  double v = W[r + q * ldw];
  for (int a = 0; a < q; ++a) v -= W[r + a * ldw] * sc->b0[a];
  R[r] = v;
}

cudaError_t launch_log_diag(const double* L, int64_t ld, int n, double* out, cudaStream_t s) {
  log_diag_kernel<<<1, 256, 0, s>>>(L, ld, n, out);
  return cudaGetLastError();
}
cudaError_t launch_col_sumsq(const double* X, int64_t ld, int n, int ncols, double* out, cudaStream_t s) {
  if (ncols <= 0) return cudaSuccess;
  col_sumsq_kernel<<<ncols, 256, 0, s>>>(X, ld, n, out);
  return cudaGetLastError();
}
cudaError_t launch_identity_cols(double* E, int n, int c0, int ncols, cudaStream_t s) {
  identity_cols_kernel<<<512, 256, 0, s>>>(E, n, c0, ncols);
  return cudaGetLastError();
}
cudaError_t launch_null_residual(const double* W, int64_t ldw, int rows, int q, const SolveConsts* sc, double* R,
                                 cudaStream_t s) {
  null_residual_kernel<<<(rows + 255) / 256, 256, 0, s>>>(W, ldw, rows, q, sc, R);
  return cudaGetLastError();
}

// The split adjoint's hand-over to the FP64 adjoint kernels: dst = (double)src
// over rows x ncols, plus shift[c] * col0 on column c when the solve ran on the
// integer-shifted SNP column x - c*1 (exact undo: L^-1 and L^-T are linear and
// col0 is the solved intercept column).
__global__ void widen_kernel(const float* __restrict__ src, int64_t lds, double* __restrict__ dst, int64_t ldd,
                             int rows, int ncols, const int8_t* __restrict__ shift, const double* __restrict__ col0) {
  const int64_t total = (int64_t)rows * ncols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / rows), r = (int)(e % rows);
    double v = (double)src[(int64_t)c * lds + r];
    if (shift) v = fma((double)shift[c], col0[r], v);
    dst[(int64_t)c * ldd + r] = v;
  }
}

cudaError_t launch_widen(const float* src, int64_t lds, double* dst, int64_t ldd, int rows, int ncols,
                         const int8_t* shift, const double* col0, cudaStream_t s) {
  if (rows <= 0 || ncols <= 0) return cudaSuccess;
  widen_kernel<<<1184, 256, 0, s>>>(src, lds, dst, ldd, rows, ncols, shift, col0);
  return cudaGetLastError();
}

}  // namespace gwas
