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
  sc->stl00 = q > 0 ? G[0] : 0.0;
}

cudaError_t launch_solve_consts(const double* G, int q, SolveConsts* sc, DevStatus* st, cudaStream_t s) {
  solve_consts_kernel<<<1, 32, 0, s>>>(G, q, sc, st);
  return cudaGetLastError();
}

// ------------------------------------------------- per-SNP reductions + solve
// acc[0..q-1] = S_BL, acc[q] = r_B, acc[QM+1] = S_BR (lane 0 after the warp reduction).
// c != 0: the sums are those of the shifted SNP x' = x - c * X_L[:, 0] (X_L[:, 0]
// the intercept).  [X_L | x'] spans the same space as [X_L | x]:  d^2 and b_p
// are unchanged, b_0 = b'_0 - c b_p, and with S = T^T S' T (T = I + c e_0 e_p^T)
// (S^-1)_00 = dSTL_0 + (g_0 + c)^2 / d^2; every other entry is unchanged.  The
// collinearity test uses the unshifted S_BR = S'_BR + 2 c S'_BL,0 + c^2 S_TL,00.
template <int QM>
__device__ __forceinline__ void solve_store(const double (&acc)[QM + 2], const SolveConsts* __restrict__ sc,
                                            int q, int col, double* __restrict__ b, double* __restrict__ se,
                                            int* __restrict__ status, double c = 0.0) {
  const int p = q + 1;
  const double sbr = acc[QM + 1], rb = acc[q];
  const double sbr_test = (c != 0.0 && q > 0) ? sbr + 2.0 * c * acc[0] + c * c * sc->stl00 : sbr;
  double l[QM > 0 ? QM : 1];
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
  if (!(d2 > SINGULAR_TAU * sbr_test)) {
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
    double v = 0.0;  // g_j = (C^-T l)_j
    for (int i = j; i < q; ++i) v = fma(sc->Cinv[i + j * QMAX], l[i], v);
    if (j == 0) v += c;
    bo[j] = sc->b0[j] - bp * v;
    if (so) so[j] = sqrt(sc->dSTL[j] + v * v / d2);
  }
  bo[q] = bp;
  if (so) so[q] = sqrt(1.0 / d2);
  if (status) status[col] = GWAS_SNP_OK;
}

template <int QM>
__device__ __forceinline__ void warp_sum(double (&acc)[QM + 2]) {
#pragma unroll
  for (int a = 0; a < QM + 2; ++a)
#pragma unroll
    for (int o = 16; o; o >>= 1) acc[a] += __shfl_xor_sync(0xffffffffu, acc[a], o);
}

// FP64 X~ (the FP64 path): FP64 products and sums.  One warp per SNP.
template <int QM>
__global__ void __launch_bounds__(256) reduce_solve_kernel(const double* __restrict__ Xt, int64_t ldt, int rows,
                                                           const double* __restrict__ W, int64_t ldw,
                                                           const SolveConsts* __restrict__ sc, int q,
                                                           int ncols, double* __restrict__ b,
                                                           double* __restrict__ se, int* __restrict__ status) {
  const int lane = threadIdx.x & 31;
  const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (col >= ncols) return;
  const double* x = Xt + (int64_t)col * ldt;
  double acc[QM + 2];
#pragma unroll
  for (int a = 0; a < QM + 2; ++a) acc[a] = 0.0;
  for (int r = lane; r < rows; r += 32) {
    const double xv = __ldcs(x + r);
#pragma unroll
    for (int a = 0; a <= QM; ++a)
      if (a <= q) acc[a] = fma(xv, W[r + a * ldw], acc[a]);
    acc[QM + 1] = fma(xv, xv, acc[QM + 1]);
  }
  warp_sum<QM>(acc);
  if (lane == 0) solve_store<QM>(acc, sc, q, col, b, se, status);
}

// FP32 X~ (the split paths).  A block takes 32 SNP columns, one per lane, and
// splits the rows into SL slices, one per warp.  Each thread streams 32-row
// runs (one 128-byte line) of its own column, the next run's loads in flight
// while the current one is summed.  The run's 32 rows of W32 (FP32,
// row-major, row stride WS) are the same for every lane: the warp loads them
// once, coalesced, into shared memory and reads them back as broadcasts.  A
// run's products are summed in FP32, runs are added with Kahan compensation
// (still FP32: B300 runs FP64 at a small fraction of the FP32 rate), and only
// the SL slice totals of a column are added in FP64, in a fixed order, so the
// result is deterministic.  Lanes past ncols read column 0 and discard it.
constexpr int RS_RUN = 32;

template <int QM, int WS, int SL>
__global__ void __launch_bounds__(32 * SL) reduce_solve_f32_kernel(
    const float* __restrict__ Xt, int64_t ldt, int rows, const float* __restrict__ W32,
    const SolveConsts* __restrict__ sc, int q, int ncols, double* __restrict__ b, double* __restrict__ se,
    int* __restrict__ status, const int8_t* __restrict__ shift) {
  constexpr int NA = QM + 2, NW4 = WS / 4, NX4 = RS_RUN / 4;
  // the W runs (inside the row loop) and the slice totals (after it) share one buffer
  constexpr int TOT_BYTES = SL * NA * 32 * 8, WSM_BYTES = SL * RS_RUN * NW4 * 16;
  __shared__ __align__(16) unsigned char smem[TOT_BYTES > WSM_BYTES ? TOT_BYTES : WSM_BYTES];
  auto tot = reinterpret_cast<double(*)[NA][32]>(smem);
  auto wsm = reinterpret_cast<float4(*)[RS_RUN * NW4]>(smem);
  const int lane = threadIdx.x & 31, slice = threadIdx.x >> 5;
  const int col = blockIdx.x * 32 + lane;
  const bool live = col < ncols;
  const float4* x4 = reinterpret_cast<const float4*>(Xt + (int64_t)(live ? col : 0) * ldt);
  const float4* w4 = reinterpret_cast<const float4*>(W32);
  float4* wmine = wsm[slice];
  float ks[NA], kc[NA];  // Kahan sum and compensation
#pragma unroll
  for (int a = 0; a < NA; ++a) ks[a] = kc[a] = 0.f;
  const int nrun = rows / RS_RUN;
  float4 xn[NX4], wn[NW4];
  if (slice < nrun) {
#pragma unroll
    for (int i = 0; i < NX4; ++i) xn[i] = __ldcs(x4 + slice * NX4 + i);
#pragma unroll
    for (int v4 = 0; v4 < NW4; ++v4) wn[v4] = __ldg(w4 + (int64_t)(slice * RS_RUN + lane) * NW4 + v4);
  }
  for (int run = slice; run < nrun; run += SL) {
    float4 xv[NX4];
#pragma unroll
    for (int i = 0; i < NX4; ++i) xv[i] = xn[i];
    __syncwarp();  // the previous run's reads of wmine are done
#pragma unroll
    for (int v4 = 0; v4 < NW4; ++v4) wmine[lane * NW4 + v4] = wn[v4];
    __syncwarp();
    const int nxt = run + SL;
    if (nxt < nrun) {
#pragma unroll
      for (int i = 0; i < NX4; ++i) xn[i] = __ldcs(x4 + nxt * NX4 + i);
#pragma unroll
      for (int v4 = 0; v4 < NW4; ++v4) wn[v4] = __ldg(w4 + (int64_t)(nxt * RS_RUN + lane) * NW4 + v4);
    }
    float part[NA];
#pragma unroll
    for (int a = 0; a < NA; ++a) part[a] = 0.f;
#pragma unroll
    for (int i = 0; i < NX4; ++i) {
      const float xs[4] = {xv[i].x, xv[i].y, xv[i].z, xv[i].w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
#pragma unroll
        for (int v4 = 0; v4 < NW4; ++v4) {
          const float4 w = wmine[(4 * i + e) * NW4 + v4];
          const float wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
          for (int t = 0; t < 4; ++t)
            if (4 * v4 + t <= QM) part[4 * v4 + t] = fmaf(xs[e], wv[t], part[4 * v4 + t]);
        }
        part[QM + 1] = fmaf(xs[e], xs[e], part[QM + 1]);
      }
    }
#pragma unroll
    for (int a = 0; a < NA; ++a) {
      const float y = part[a] - kc[a];
      const float t = ks[a] + y;
      kc[a] = (t - ks[a]) - y;
      ks[a] = t;
    }
  }
  __syncthreads();  // every warp is done with its W runs
#pragma unroll
  for (int a = 0; a < NA; ++a) tot[slice][a][lane] = (double)ks[a] - (double)kc[a];
  __syncthreads();
  if (slice != 0 || !live) return;
  double sum[NA];
#pragma unroll
  for (int a = 0; a < NA; ++a) {
    double t = tot[0][a][lane];
    for (int s2 = 1; s2 < SL; ++s2) t += tot[s2][a][lane];
    sum[a] = t;
  }
  solve_store<QM>(sum, sc, q, col, b, se, status, shift ? (double)shift[col] : 0.0);
}

// FP32 X~, few covariates (q <= 7): a block takes RC SNP columns and splits
// the rows into RW slices of whole 128-row chunks, one slice per warp.  Lane l
// covers rows 4l .. 4l+3 of a chunk, so every float4 load of a column is one
// coalesced 512-byte segment, and the four W32 rows it needs come from L1.
// A chunk's products are summed in FP32, chunks are added with Kahan
// compensation (FP32), a warp's lanes are added in FP64 by a butterfly and the
// RW slice totals of a column in FP64, in a fixed order (deterministic).
// Lanes past ncols re-read the last column and discard the result.
constexpr int RC_RW = 4;  // row slices (warps) per block

template <int QM, int WS, int RC>
__global__ void __launch_bounds__(32 * RC_RW) reduce_solve_f32c_kernel(
    const float* __restrict__ Xt, int64_t ldt, int rows, const float* __restrict__ W32,
    const SolveConsts* __restrict__ sc, int q, int ncols, double* __restrict__ b, double* __restrict__ se,
    int* __restrict__ status, const int8_t* __restrict__ shift) {
  constexpr int NA = QM + 2, NW4 = WS / 4;
  __shared__ double tot[RC_RW][RC][NA];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nchunk = rows >> 7;
  const int t0 = w * nchunk / RC_RW, t1 = (w + 1) * nchunk / RC_RW;
  const float4* w4 = reinterpret_cast<const float4*>(W32);
  const int col0 = blockIdx.x * RC;
  const float4* xp[RC];
#pragma unroll
  for (int c = 0; c < RC; ++c) {
    const int col = col0 + c < ncols ? col0 + c : ncols - 1;
    xp[c] = reinterpret_cast<const float4*>(Xt + (int64_t)col * ldt) + lane;
  }
  float ks[RC][NA], kc[RC][NA];
#pragma unroll
  for (int c = 0; c < RC; ++c)
#pragma unroll
    for (int a = 0; a < NA; ++a) ks[c][a] = kc[c][a] = 0.f;
  float4 xn[RC];
  if (t0 < t1) {
#pragma unroll
    for (int c = 0; c < RC; ++c) xn[c] = __ldcs(xp[c] + t0 * 32);
  }
  for (int t = t0; t < t1; ++t) {
    float4 xv[RC];
#pragma unroll
    for (int c = 0; c < RC; ++c) xv[c] = xn[c];
    if (t + 1 < t1) {
#pragma unroll
      for (int c = 0; c < RC; ++c) xn[c] = __ldcs(xp[c] + (t + 1) * 32);
    }
    float4 wv[4][NW4];
    const int64_t r0 = (int64_t)t * 128 + 4 * lane;
#pragma unroll
    for (int rr = 0; rr < 4; ++rr)
#pragma unroll
      for (int v4 = 0; v4 < NW4; ++v4) wv[rr][v4] = __ldg(w4 + (r0 + rr) * NW4 + v4);
#pragma unroll
    for (int c = 0; c < RC; ++c) {
      const float xs[4] = {xv[c].x, xv[c].y, xv[c].z, xv[c].w};
      float part[NA];
#pragma unroll
      for (int a = 0; a < NA; ++a) part[a] = 0.f;
#pragma unroll
      for (int rr = 0; rr < 4; ++rr) {
#pragma unroll
        for (int v4 = 0; v4 < NW4; ++v4) {
          const float wr[4] = {wv[rr][v4].x, wv[rr][v4].y, wv[rr][v4].z, wv[rr][v4].w};
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (4 * v4 + e <= QM) part[4 * v4 + e] = fmaf(xs[rr], wr[e], part[4 * v4 + e]);
        }
        part[QM + 1] = fmaf(xs[rr], xs[rr], part[QM + 1]);
      }
#pragma unroll
      for (int a = 0; a < NA; ++a) {
        const float y = part[a] - kc[c][a];
        const float s2 = ks[c][a] + y;
        kc[c][a] = (s2 - ks[c][a]) - y;
        ks[c][a] = s2;
      }
    }
  }
#pragma unroll
  for (int c = 0; c < RC; ++c)
#pragma unroll
    for (int a = 0; a < NA; ++a) {
      double v = (double)ks[c][a] - (double)kc[c][a];
#pragma unroll
      for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) tot[w][c][a] = v;
    }
  __syncthreads();
  if (threadIdx.x < RC && col0 + (int)threadIdx.x < ncols) {
    const int c = threadIdx.x, col = col0 + c;
    double sum[NA];
#pragma unroll
    for (int a = 0; a < NA; ++a) {
      double v = tot[0][c][a];
      for (int s2 = 1; s2 < RC_RW; ++s2) v += tot[s2][c][a];
      sum[a] = v;
    }
    solve_store<QM>(sum, sc, q, col, b, se, status, shift ? (double)shift[col] : 0.0);
  }
}

cudaError_t launch_reduce_solve(const void* Xt, XtKind kind, int64_t ldt, int rows, const double* W,
                                int64_t ldw, const SolveConsts* sc, int q, int ncols, double* b, double* se,
                                int* status, cudaStream_t s, const float* W32, const int8_t* shift) {
  if (ncols <= 0) return cudaSuccess;
  const int grid = (ncols + 7) / 8;
  if (kind == XT_F64) {
    const double* X = static_cast<const double*>(Xt);
    if (q <= 3)
      reduce_solve_kernel<3><<<grid, 256, 0, s>>>(X, ldt, rows, W, ldw, sc, q, ncols, b, se, status);
    else if (q <= 7)
      reduce_solve_kernel<7><<<grid, 256, 0, s>>>(X, ldt, rows, W, ldw, sc, q, ncols, b, se, status);
    else
      reduce_solve_kernel<QMAX><<<grid, 256, 0, s>>>(X, ldt, rows, W, ldw, sc, q, ncols, b, se, status);
    return cudaGetLastError();
  }
  if (!W32) return cudaErrorInvalidValue;
  const float* X = static_cast<const float*>(Xt);
  if ((rows % RS_RUN) || (ldt % RS_RUN)) return cudaErrorInvalidValue;  // whole 128-byte runs
  const int g32 = (ncols + 31) / 32;
  if (q <= 3 && rows % 128 == 0)
    reduce_solve_f32c_kernel<3, 4, 4><<<(ncols + 3) / 4, 32 * RC_RW, 0, s>>>(X, ldt, rows, W32, sc, q, ncols, b, se,
                                                                            status, shift);
  else if (q <= 3)
    reduce_solve_f32_kernel<3, 4, 16><<<g32, 512, 0, s>>>(X, ldt, rows, W32, sc, q, ncols, b, se, status, shift);
  else if (q <= 7 && rows % 128 == 0)
    reduce_solve_f32c_kernel<7, 8, 2><<<(ncols + 1) / 2, 32 * RC_RW, 0, s>>>(X, ldt, rows, W32, sc, q, ncols, b, se,
                                                                            status, shift);
  else if (q <= 7)
    reduce_solve_f32_kernel<7, 8, 16><<<g32, 512, 0, s>>>(X, ldt, rows, W32, sc, q, ncols, b, se, status, shift);
  else
    reduce_solve_f32_kernel<QMAX, 16, 8><<<g32, 256, 0, s>>>(X, ldt, rows, W32, sc, q, ncols, b, se, status, shift);
  return cudaGetLastError();
}

// W32 = W in FP32, row-major with row stride w32_stride(q) (zero-padded).
__global__ void make_w32_kernel(const double* __restrict__ W, int64_t ldw, int rows, int nc, int ws,
                                float* __restrict__ W32) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)rows * ws;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / ws), a = (int)(e % ws);
    W32[e] = a < nc ? (float)W[r + a * ldw] : 0.f;
  }
}

int w32_stride(int q) { return q <= 3 ? 4 : (q <= 7 ? 8 : 16); }

cudaError_t launch_make_w32(const double* W, int64_t ldw, int rows, int q, float* W32, cudaStream_t s) {
  make_w32_kernel<<<256, 256, 0, s>>>(W, ldw, rows, q + 1, w32_stride(q), W32);
  return cudaGetLastError();
}

}  // namespace gwas
