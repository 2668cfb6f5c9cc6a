// a3, a7, a8: the FP64 reductions of Listing 1 and the per-SNP p x p solve.
//
// Loop-invariant part (once per study):  W = [X~_L | y~],
//     G = W^T W  gives  S_TL = X~_L^T X~_L  and  r_T = X~_L^T y~.
// Per SNP i (loop body of Listing 1):
//     S_BL = x~_i^T X~_L,  S_BR = x~_i^T x~_i,  r_B = x~_i^T y~,
//     S = [S_TL S_BL^T; S_BL S_BR],  r~ = [r_T; r_B],  b = S^-1 r~ (posv).
// The solve uses the block Cholesky factor of S.  With S_TL = C C^T:
//     l = C^-1 S_BL^T,   d^2 = S_BR - l^T l,
//     b_p = (r_B - l^T zT) / d^2,  g = C^-T l,  b_T = b0 - b_p g,
//     se_T^2 = dSTL + g^2 / d^2,  se_p^2 = 1 / d^2,
// where zT = C^-1 r_T, b0 = S_TL^-1 r_T and dSTL = diag(S_TL^-1) are the
// SolveConsts.  A SNP with d^2 <= SINGULAR_TAU * S_BR is numerically
// collinear with X_L: status GWAS_SNP_SINGULAR and NaN outputs.
#include "gwas_internal.cuh"

namespace gwas {

// ------------------------------------------------------------ G = W^T W
__global__ void __launch_bounds__(256) gram_kernel(const double* __restrict__ W, int64_t ldw, int rows, int nc,
                                                   double* __restrict__ G) {
  const int a = blockIdx.x, b = blockIdx.y;
  if (b > a) return;
  __shared__ double red[8];
  double s = 0.0;
  for (int r = threadIdx.x; r < rows; r += blockDim.x) s = fma(W[r + a * ldw], W[r + b * ldw], s);
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    G[a + b * nc] = t;
    G[b + a * nc] = t;
  }
}

cudaError_t launch_gram(const double* W, int64_t ldw, int rows, int nc, double* G, cudaStream_t s) {
  gram_kernel<<<dim3(nc, nc), 256, 0, s>>>(W, ldw, rows, nc, G);
  return cudaGetLastError();
}

// ------------------------------------------------------------ solve constants
__global__ void solve_consts_kernel(const double* __restrict__ G, int q, SolveConsts* sc, DevStatus* st) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int nc = q + 1;
  double C[QMAX * QMAX];
  sc->q = q;
  for (int i = 0; i < QMAX * QMAX; ++i) { C[i] = 0.0; sc->Cinv[i] = 0.0; }
  // Cholesky of S_TL = G[0:q, 0:q]
  for (int j = 0; j < q; ++j) {
    double d = G[j + j * nc];
    for (int t = 0; t < j; ++t) d -= C[j + t * QMAX] * C[j + t * QMAX];
    if (!(d > SINGULAR_TAU * G[j + j * nc])) { st->sc_err = 1; return; }
    d = sqrt(d);
    C[j + j * QMAX] = d;
    for (int i = j + 1; i < q; ++i) {
      double v = G[i + j * nc];
      for (int t = 0; t < j; ++t) v -= C[i + t * QMAX] * C[j + t * QMAX];
      C[i + j * QMAX] = v / d;
    }
  }
  // Cinv = C^-1 (lower), column by column
  for (int c = 0; c < q; ++c) {
    for (int i = 0; i < q; ++i) {
      if (i < c) continue;
      double v = (i == c) ? 1.0 : 0.0;
      for (int t = c; t < i; ++t) v -= C[i + t * QMAX] * sc->Cinv[t + c * QMAX];
      sc->Cinv[i + c * QMAX] = v / C[i + i * QMAX];
    }
  }
  // zT = C^-1 r_T,  b0 = C^-T zT,  dSTL_j = sum_i Cinv_ij^2
  for (int i = 0; i < q; ++i) {
    double v = 0.0;
    for (int t = 0; t <= i; ++t) v += sc->Cinv[i + t * QMAX] * G[t + q * nc];
    sc->zT[i] = v;
  }
  for (int j = 0; j < q; ++j) {
    double v = 0.0, d = 0.0;
    for (int i = j; i < q; ++i) {
      v += sc->Cinv[i + j * QMAX] * sc->zT[i];
      d += sc->Cinv[i + j * QMAX] * sc->Cinv[i + j * QMAX];
    }
    sc->b0[j] = v;
    sc->dSTL[j] = d;
  }
}

cudaError_t launch_solve_consts(const double* G, int q, SolveConsts* sc, DevStatus* st, cudaStream_t s) {
  solve_consts_kernel<<<1, 32, 0, s>>>(G, q, sc, st);
  return cudaGetLastError();
}

// ------------------------------------------------- per-SNP reductions + solve
template <typename T>
__device__ __forceinline__ double load_x(const T* p) { return (double)__ldcs(p); }

// One warp per SNP.  QM is a compile-time bound on q (accumulators in registers).
template <int QM, typename T>
__global__ void __launch_bounds__(256) reduce_solve_kernel(const T* __restrict__ Xt, int64_t ldt, int rows,
                                                           const double* __restrict__ W, int64_t ldw,
                                                           const SolveConsts* __restrict__ sc, int q,
                                                           int ncols, double* __restrict__ b,
                                                           double* __restrict__ se, int* __restrict__ status) {
  const int lane = threadIdx.x & 31;
  const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (col >= ncols) return;
  const T* x = Xt + (int64_t)col * ldt;
  double acc[QM + 2];  // [0..q-1] S_BL, [q] r_B, [q+1] S_BR
#pragma unroll
  for (int a = 0; a < QM + 2; ++a) acc[a] = 0.0;
  for (int r = lane; r < rows; r += 32) {
    const double xv = load_x(x + r);
#pragma unroll
    for (int a = 0; a <= QM; ++a)
      if (a <= q) acc[a] = fma(xv, W[r + a * ldw], acc[a]);
    acc[QM + 1] = fma(xv, xv, acc[QM + 1]);
  }
#pragma unroll
  for (int a = 0; a < QM + 2; ++a)
#pragma unroll
    for (int o = 16; o; o >>= 1) acc[a] += __shfl_xor_sync(0xffffffffu, acc[a], o);
  if (lane != 0) return;

  const int p = q + 1;
  const double sbr = acc[QM + 1], rb = acc[q];
  double l[QM > 0 ? QM : 1], g[QM > 0 ? QM : 1];
  double ll = 0.0, lz = 0.0;
#pragma unroll
  for (int i = 0; i < QM; ++i) {
    if (i >= q) break;
    double v = 0.0;
    for (int t = 0; t <= i; ++t) v = fma(sc->Cinv[i + t * QMAX], acc[t], v);
    l[i] = v;
    ll = fma(v, v, ll);
    lz = fma(v, sc->zT[i], lz);
  }
  const double d2 = sbr - ll;
  double* bo = b + (int64_t)col * p;
  double* so = se ? se + (int64_t)col * p : nullptr;
  if (!(d2 > SINGULAR_TAU * sbr)) {
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    for (int j = 0; j < p; ++j) {
      bo[j] = nan;
      if (so) so[j] = nan;
    }
    if (status) status[col] = GWAS_SNP_SINGULAR;
    return;
  }
  const double bp = (rb - lz) / d2;
#pragma unroll
  for (int j = 0; j < QM; ++j) {
    if (j >= q) break;
    double v = 0.0;
    for (int i = j; i < q; ++i) v = fma(sc->Cinv[i + j * QMAX], l[i], v);
    g[j] = v;
    bo[j] = sc->b0[j] - bp * v;
    if (so) so[j] = sqrt(sc->dSTL[j] + v * v / d2);
  }
  bo[q] = bp;
  if (so) so[q] = sqrt(1.0 / d2);
  if (status) status[col] = GWAS_SNP_OK;
  (void)g;
}

template <typename T>
static cudaError_t dispatch_rs(const T* Xt, int64_t ldt, int rows, const double* W, int64_t ldw,
                               const SolveConsts* sc, int q, int ncols, double* b, double* se, int* status,
                               cudaStream_t s) {
  const int grid = (ncols + 7) / 8;
  if (q <= 3)
    reduce_solve_kernel<3, T><<<grid, 256, 0, s>>>(Xt, ldt, rows, W, ldw, sc, q, ncols, b, se, status);
  else if (q <= 7)
    reduce_solve_kernel<7, T><<<grid, 256, 0, s>>>(Xt, ldt, rows, W, ldw, sc, q, ncols, b, se, status);
  else
    reduce_solve_kernel<QMAX, T><<<grid, 256, 0, s>>>(Xt, ldt, rows, W, ldw, sc, q, ncols, b, se, status);
  return cudaGetLastError();
}

cudaError_t launch_reduce_solve(const void* Xt, XtKind kind, int64_t ldt, int rows, const double* W,
                                int64_t ldw, const SolveConsts* sc, int q, int ncols, double* b, double* se,
                                int* status, cudaStream_t s) {
  if (ncols <= 0) return cudaSuccess;
  if (kind == XT_F64)
    return dispatch_rs(static_cast<const double*>(Xt), ldt, rows, W, ldw, sc, q, ncols, b, se, status, s);
  return dispatch_rs(static_cast<const float*>(Xt), ldt, rows, W, ldw, sc, q, ncols, b, se, status, s);
}

}  // namespace gwas
