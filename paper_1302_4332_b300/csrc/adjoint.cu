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
#include <cuda_fp16.h>

#include "gwas_internal.cuh"
#include "tc_ptx.cuh"

namespace gwas {

// The per-SNP adjoint from the forward sums af (x~ against [X~_L | y~], then
// x~ . x~) and the transpose sums ah (the same for x^ against [X^_L | y^]).
template <int QM>
__device__ __forceinline__ void adjoint_store(const double (&af)[QM + 2], const double (&ah)[QM + 2],
                                              const SolveConsts* __restrict__ sc, const double* __restrict__ GH,
                                              int q, int col, double h, double sigma2, double* __restrict__ chi2,
                                              double* __restrict__ dh, double* __restrict__ wv) {
  const int p = q + 1, nc = q + 1;
  // forward: l = C^-1 S_BL, d^2, b, g = C^-T l (as in the block solve)
  double l[QM > 0 ? QM : 1], g[QM > 0 ? QM : 1];
  double ll = 0.0, lz = 0.0;
  for (int i = 0; i < q; ++i) {
    double v = 0.0;
    for (int t = 0; t <= i; ++t) v = fma(sc->Cinv[i + t * QMAX], af[t], v);
    l[i] = v;
    ll = fma(v, v, ll);
    lz = fma(v, sc->zT[0][i], lz);
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
    bT[j] = sc->b0[0][j] - bp * v;
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
  adjoint_store<QM>(af, ah, sc, GH, q, col, h, sigma2, chi2, dh, wv);
}

// The split precisions' adjoint from the exact products C = A x' of
// exact_products.cu (A: three slabs of RS rows, slab k = slice k of W's rows,
// then slices k and k + 3 of the ne = 2(q+1) appended rows [X^_L | y^ |
// W X^_L | W y^]^T): one warp per SNP column.  Over W's rows r < n, with the
// integers x'_r and c_k = C[k RS + r]:
//   P_k = sum_r x'_r c_k  (int64, exact),  S_BR = x'^T W x' = (P_1 + 2^-10 P_2 + 2^-20 P_3) / s_W,
//   ||x^'||^2 = sum_r u_r^2 / s_W^2,  u_r = c_1 + 2^-10 c_2 + 2^-20 c_3  (exact; the sum of squares too
//   for dosage-sized values -- its relative error reaches the gradient amplified by the cancellation
//   in ||W a||^2, so an FP32 sum would not do),
// and appended row e gives sum_k 2^-10k C[...] / s_e (six slices), the
// forward sums x'^T [X^_L | y^] and the transpose sums x^'^T [X^_L | y^].
// Then the p x p adjoint as in the FP64 path.
template <int QM>
__global__ void __launch_bounds__(256) exact_adjoint_kernel(
    const int32_t* __restrict__ C, int64_t ldc, int RS, const __half* __restrict__ xc, int64_t ldx, int n, int n_pad,
    int ne, const double* __restrict__ inv_scale, const SolveConsts* __restrict__ sc, const double* __restrict__ GH,
    int q, int ncols, double h, double sigma2, const int* __restrict__ xmax, double* __restrict__ chi2,
    double* __restrict__ dh, double* __restrict__ wv) {
  const int lane = threadIdx.x & 31;
  const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (col >= ncols) return;
  const bool small44 = 512LL * (*xmax) * n_pad <= (1LL << 24);
  const int32_t* cc = C + (int64_t)col * ldc;
  const __half* x = xc + (int64_t)col * ldx;
  // P_k: exact in int64 (|x'_r c_k| < 2^39).  ||x^'||^2 = 2^-40 sum_r T_r^2 with
  // T_r = 2^20 c_1 + 2^10 c_2 + c_3 (an integer): when |T_r| < 2^44 (small44:
  // 512 * max|x'| * n_pad <= 2^24, e.g. dosages and n <= 16,384), exact as
  // T = 2^22 t_h + t_l, T^2 = 2^44 t_h^2 + 2^23 t_h t_l + t_l^2, each part an
  // int64 sum; otherwise T_r^2 summed in FP64.
  long long p1 = 0, p2 = 0, p3 = 0, shh = 0, shl = 0, sll = 0;
  double qq = 0.0;
  auto row = [&](int xi, int a1, int a2, int a3) {
    p1 += (long long)xi * a1;
    p2 += (long long)xi * a2;
    p3 += (long long)xi * a3;
    const long long T = ((long long)a1 << 20) + ((long long)a2 << 10) + a3;
    if (small44) {  // |t_h| <= 2^23, 0 <= t_l < 2^22: 32 x 32 -> 64-bit products
      const int th = (int)(T >> 22), tl = (int)(T & 0x3FFFFF);
      shh += (long long)th * th;
      shl += (long long)th * tl;
      sll += (long long)tl * tl;
    } else {
      const double u = (double)T;
      qq = fma(u, u, qq);
    }
  };
  // four rows a lane per step: 16-byte loads of each slab's products and 8 of
  // x' (C's rows are 16-byte aligned: ldc and RS are multiples of 256, and
  // x''s of 8: ldx = n_pad).  Rows n .. n_pad - 1 add nothing: x' is 0 there
  // and so are the products (W is zero on the padding).
  const int4* c1 = reinterpret_cast<const int4*>(cc);
  const int4* c2 = reinterpret_cast<const int4*>(cc + RS);
  const int4* c3 = reinterpret_cast<const int4*>(cc + 2 * RS);
  const uint2* x4 = reinterpret_cast<const uint2*>(x);
#pragma unroll 2
  for (int r4 = lane; r4 < (n_pad >> 2); r4 += 32) {
    const int4 A1 = __ldcs(c1 + r4), A2 = __ldcs(c2 + r4), A3 = __ldcs(c3 + r4);
    const uint2 xv = __ldg(x4 + r4);
    const __half2 h01 = *reinterpret_cast<const __half2*>(&xv.x);
    const __half2 h23 = *reinterpret_cast<const __half2*>(&xv.y);
    row(__half2int_rn(__low2half(h01)), A1.x, A2.x, A3.x);
    row(__half2int_rn(__high2half(h01)), A1.y, A2.y, A3.y);
    row(__half2int_rn(__low2half(h23)), A1.z, A2.z, A3.z);
    row(__half2int_rn(__high2half(h23)), A1.w, A2.w, A3.w);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    p1 += __shfl_xor_sync(0xffffffffu, p1, o);
    p2 += __shfl_xor_sync(0xffffffffu, p2, o);
    p3 += __shfl_xor_sync(0xffffffffu, p3, o);
    if (small44) {
      shh += __shfl_xor_sync(0xffffffffu, shh, o);
      shl += __shfl_xor_sync(0xffffffffu, shl, o);
      sll += __shfl_xor_sync(0xffffffffu, sll, o);
    } else {
      qq += __shfl_xor_sync(0xffffffffu, qq, o);
    }
  }
  if (small44) qq = fma((double)shh, 0x1p44, fma((double)shl, 0x1p23, (double)sll));
  qq *= 0x1p-40;
  // appended row `lane` (< ne): six slices, the smallest first
  double ev = 0.0;
  if (lane < ne) {
    const int r0 = n_pad + lane, r1 = n_pad + ne + lane;
    double v = 0.0;
    v = fma((double)cc[2 * RS + r1], 0x1p-50, v);
    v = fma((double)cc[RS + r1], 0x1p-40, v);
    v = fma((double)cc[r1], 0x1p-30, v);
    v = fma((double)cc[2 * RS + r0], 0x1p-20, v);
    v = fma((double)cc[RS + r0], 0x1p-10, v);
    ev = ((double)cc[r0] + v) * inv_scale[1 + lane];
  }
  double evs[2 * (QM + 1)];
#pragma unroll
  for (int e = 0; e < 2 * (QM + 1); ++e) evs[e] = __shfl_sync(0xffffffffu, ev, e < 32 ? e : 0);
  if (lane != 0) return;
  const double is = inv_scale[0];
  double af[QM + 2], ah[QM + 2];
#pragma unroll
  for (int a = 0; a < QM + 2; ++a) af[a] = ah[a] = 0.0;
  for (int a = 0; a <= q; ++a) {
    af[a] = evs[a];          // x'^T X^_L, x'^T y^
    ah[a] = evs[q + 1 + a];  // x^'^T X^_L, x^'^T y^
  }
  af[QM + 1] = fma((double)p3, 0x1p-20, fma((double)p2, 0x1p-10, (double)p1)) * is;
  ah[QM + 1] = qq * is * is;
  adjoint_store<QM>(af, ah, sc, GH, q, col, h, sigma2, chi2, dh, wv);
}

// Block a (< q + 1): quantity a over the SNPs -- uT[a] for a < q, the block's
// d chi2/dh (added to *dh_accum) for a = q -- 256 threads each over a strided
// slice, then a fixed tree in shared memory (deterministic).
__global__ void __launch_bounds__(256) adjoint_sum_kernel(const double* __restrict__ dh, const double* __restrict__ wv,
                                                          int q, int ncols, double* __restrict__ dh_accum,
                                                          double* __restrict__ uT) {
  __shared__ double red[256];
  const int a = blockIdx.x;
  double s0 = 0.0, s1 = 0.0;
  int i = threadIdx.x;
  for (; i + 256 < ncols; i += 512) {  // two loads in flight per thread
    s0 += (a == q) ? dh[i] : wv[(int64_t)i * (q + 1) + a];
    s1 += (a == q) ? dh[i + 256] : wv[(int64_t)(i + 256) * (q + 1) + a];
  }
  if (i < ncols) s0 += (a == q) ? dh[i] : wv[(int64_t)i * (q + 1) + a];
  red[threadIdx.x] = s0 + s1;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (a == q)
      *dh_accum += red[0];
    else
      uT[a] = red[0];
  }
}

// dy[r] += sum_a uT[a] X^_L[r, a] + sum_i w_p,i x^_i[r]   (r < n), in two
// steps so that the SNP sum spreads over the SMs: part[k][r] = the sum over
// SNP chunk k (DY_CHUNK columns), then the chunks in order.
constexpr int DY_CHUNK = 128;

__global__ void adjoint_dy_part_kernel(const double* __restrict__ Xh, int64_t ldt, const double* __restrict__ wv,
                                       int q, int n, int ncols, double* __restrict__ part) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int i0 = blockIdx.y * DY_CHUNK, i1 = i0 + DY_CHUNK < ncols ? i0 + DY_CHUNK : ncols;
  double s = 0.0;
  for (int i = i0; i < i1; ++i) s = fma(wv[(int64_t)i * (q + 1) + q], Xh[r + (int64_t)i * ldt], s);
  part[(int64_t)blockIdx.y * n + r] = s;
}

__global__ void adjoint_dy_sum_kernel(const double* __restrict__ Wh, int64_t ldw, const double* __restrict__ uT,
                                      int q, int n, int nchunks, const double* __restrict__ part,
                                      double* __restrict__ dy) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double s = 0.0;
  for (int a = 0; a < q; ++a) s = fma(uT[a], Wh[r + a * ldw], s);
  for (int k = 0; k < nchunks; ++k) s += part[(int64_t)k * n + r];
  dy[r] += s;
}

int adjoint_dy_chunks(int bs) { return (bs + DY_CHUNK - 1) / DY_CHUNK; }




cudaError_t launch_adjoint(const double* Xt, const double* Xh, int64_t ldt, int rows, int n, const double* W,
                           const double* Wh, int64_t ldw, const SolveConsts* sc, const double* GH, int q,
                           int ncols, double h, double sigma2, double* chi2, double* dh, double* wv, double* uT,
                           double* dh_accum, double* dy_accum, double* dy_part, cudaStream_t s) {
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
  adjoint_sum_kernel<<<q + 1, 256, 0, s>>>(dh, wv, q, ncols, dh_accum, uT);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int nchunks = adjoint_dy_chunks(ncols);
  adjoint_dy_part_kernel<<<dim3((n + 255) / 256, nchunks), 256, 0, s>>>(Xh, ldt, wv, q, n, ncols, dy_part);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  adjoint_dy_sum_kernel<<<(n + 255) / 256, 256, 0, s>>>(Wh, ldw, uT, q, n, nchunks, dy_part, dy_accum);
  return cudaGetLastError();
}

cudaError_t launch_exact_adjoint_sums(const int32_t* C, int64_t ldc, int RS, const __half* xc, int64_t ldx, int n,
                                      int n_pad, int ne, const double* inv_scale, const SolveConsts* sc,
                                      const double* GH, int q, int ncols, double h, double sigma2, const int* xmax,
                                      double* chi2, double* dh, double* wv, double* dh_accum, double* uT,
                                      cudaStream_t s) {
  if (ncols <= 0) return cudaSuccess;
  if (ne != 2 * (q + 1) || ne > 32) return cudaErrorInvalidValue;
  const int grid = (ncols + 7) / 8;
  if (q <= 3)
    exact_adjoint_kernel<3><<<grid, 256, 0, s>>>(C, ldc, RS, xc, ldx, n, n_pad, ne, inv_scale, sc, GH, q, ncols, h,
                                                 sigma2, xmax, chi2, dh, wv);
  else if (q <= 7)
    exact_adjoint_kernel<7><<<grid, 256, 0, s>>>(C, ldc, RS, xc, ldx, n, n_pad, ne, inv_scale, sc, GH, q, ncols, h,
                                                 sigma2, xmax, chi2, dh, wv);
  else
    exact_adjoint_kernel<QMAX><<<grid, 256, 0, s>>>(C, ldc, RS, xc, ldx, n, n_pad, ne, inv_scale, sc, GH, q, ncols,
                                                    h, sigma2, xmax, chi2, dh, wv);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  adjoint_sum_kernel<<<q + 1, 256, 0, s>>>(dh, wv, q, ncols, dh_accum, uT);
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
  for (int a = 0; a < q; ++a) v -= W[r + a * ldw] * sc->b0[0][a];
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

}  // namespace gwas
