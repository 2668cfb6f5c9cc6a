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
#include "tc_ptx.cuh"

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
__global__ void solve_consts_kernel(const double* __restrict__ G, int q, int t, SolveConsts* sc, DevStatus* st) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int nc = q + t;  // G = W^T W over [X~_L | Y~]
  double C[QMAX * QMAX];
  sc->q = q;
  sc->t = t;
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
  // per phenotype k: zT = C^-1 r_T,  b0 = C^-T zT;  dSTL_j = sum_i Cinv_ij^2
  for (int k = 0; k < t; ++k) {
    for (int i = 0; i < q; ++i) {
      double v = 0.0;
      for (int u = 0; u <= i; ++u) v += sc->Cinv[i + u * QMAX] * G[u + (q + k) * nc];
      sc->zT[k][i] = v;
    }
    for (int j = 0; j < q; ++j) {
      double v = 0.0;
      for (int i = j; i < q; ++i) v += sc->Cinv[i + j * QMAX] * sc->zT[k][i];
      sc->b0[k][j] = v;
    }
  }
  for (int j = 0; j < q; ++j) {
    double d = 0.0;
    for (int i = j; i < q; ++i) d += sc->Cinv[i + j * QMAX] * sc->Cinv[i + j * QMAX];
    sc->dSTL[j] = d;
  }
  sc->stl00 = q > 0 ? G[0] : 0.0;
}

cudaError_t launch_solve_consts(const double* G, int q, int t, SolveConsts* sc, DevStatus* st, cudaStream_t s) {
  solve_consts_kernel<<<1, 32, 0, s>>>(G, q, t, sc, st);
  return cudaGetLastError();
}

// ------------------------------------------------- per-SNP reductions + solve
// acc[0..q-1] = S_BL, acc[q + k] = r_B of phenotype k (k < t), acc[QM+1] = S_BR
// (QM >= q + t - 1).  S, hence d^2, se and the status, is the same for every
// phenotype; b of phenotype k goes to b + k * bstride.
// c != 0: the sums are those of the shifted SNP x' = x - c * X_L[:, 0] (X_L[:, 0]
// the intercept).  [X_L | x'] spans the same space as [X_L | x]:  d^2 and b_p
// are unchanged, b_0 = b'_0 - c b_p, and with S = T^T S' T (T = I + c e_0 e_p^T)
// (S^-1)_00 = dSTL_0 + (g_0 + c)^2 / d^2; every other entry is unchanged.  The
// collinearity test uses the unshifted S_BR = S'_BR + 2 c S'_BL,0 + c^2 S_TL,00.
template <int QM>
__device__ __forceinline__ void solve_store(const double (&acc)[QM + 2], const SolveConsts* __restrict__ sc,
                                            int q, int col, double* __restrict__ b, double* __restrict__ se,
                                            int* __restrict__ status, double c = 0.0, int t = 1,
                                            int64_t bstride = 0) {
  const int p = q + 1;
  const double sbr = acc[QM + 1];
  const double sbr_test = (c != 0.0 && q > 0) ? sbr + 2.0 * c * acc[0] + c * c * sc->stl00 : sbr;
  double l[QM > 0 ? QM : 1];
  double ll = 0.0;
#pragma unroll
  for (int i = 0; i < QM; ++i) {  // compile-time indices keep l and g in registers
    double v = 0.0;
#pragma unroll
    for (int u = 0; u <= i; ++u) v = fma(sc->Cinv[i + u * QMAX], acc[u], v);
    l[i] = i < q ? v : 0.0;
    ll = fma(l[i], l[i], ll);
  }
  const double d2 = sbr - ll;
  double* so = se ? se + (int64_t)col * p : nullptr;
  if (!(d2 > SINGULAR_TAU * sbr_test)) {
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    for (int k = 0; k < t; ++k)
      for (int j = 0; j < p; ++j) b[k * bstride + (int64_t)col * p + j] = nan;
    if (so)
      for (int j = 0; j < p; ++j) so[j] = nan;
    if (status) status[col] = GWAS_SNP_SINGULAR;
    return;
  }
  const double rd2 = 1.0 / d2;  // one division: the chain of FP64 operations per SNP is the solve's latency
  double g[QM > 0 ? QM : 1];    // g = C^-T l (+ c e_0: the shift)
#pragma unroll
  for (int j = 0; j < QM; ++j) {
    double v = 0.0;
#pragma unroll
    for (int i = j; i < QM; ++i) v = fma(sc->Cinv[i + j * QMAX], l[i], v);  // l[i] = 0 for i >= q
    if (j == 0) v += c;
    g[j] = v;
    if (so && j < q) so[j] = sqrt(sc->dSTL[j] + v * v * rd2);
  }
  if (so) so[q] = sqrt(rd2);
  for (int k = 0; k < t; ++k) {
    double lz = 0.0;
#pragma unroll
    for (int i = 0; i < QM; ++i) lz = fma(l[i], sc->zT[k][i], lz);
    double rb = 0.0;  // acc[q + k] without a run-time index (which would put acc in local memory)
#pragma unroll
    for (int a = 0; a <= QM; ++a)
      if (a == q + k) rb = acc[a];
    const double bp = (rb - lz) * rd2;
    double* bo = b + k * bstride + (int64_t)col * p;
#pragma unroll
    for (int j = 0; j < QM; ++j)
      if (j < q) bo[j] = sc->b0[k][j] - bp * g[j];
    bo[q] = bp;
  }
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
                                                           double* __restrict__ se, int* __restrict__ status, int t,
                                                           int64_t bstride) {
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
      if (a < q + t) acc[a] = fma(xv, W[r + a * ldw], acc[a]);
    acc[QM + 1] = fma(xv, xv, acc[QM + 1]);
  }
  warp_sum<QM>(acc);
  if (lane == 0) solve_store<QM>(acc, sc, q, col, b, se, status, 0.0, t, bstride);
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
    int* __restrict__ status, const int8_t* __restrict__ shift, int t, int64_t bstride) {
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
  solve_store<QM>(sum, sc, q, col, b, se, status, shift ? (double)shift[col] : 0.0, t, bstride);
}

// FP32 X~ streamed by TMA (the split paths, q <= 7).  A persistent block takes
// a contiguous range of SNP columns in groups of BG; one producer thread
// streams each group in chunks of BCH rows -- two tiled loads of 256 rows x
// 32 columns (32 KB each) and one bulk copy of the chunk's W32 rows -- into
// shared-memory stages completing on the stage's mbarrier, so a block keeps
// ~150-200 KB of loads in flight without holding them in registers.  Consumer warp w owns columns 2w and 2w+1 of the
// group (one load of a W row serves both); in each 128-row sub-chunk lane l
// takes rows 32r + l (r = 0..3), so its shared-memory loads are
// conflict-free.  Sums: FP32 over a chunk (16 rows per lane), Kahan across
// chunks, across the lanes a fixed butterfly in double-FP32 (error-free
// TwoSum steps; FP64 arithmetic is a small fraction of the FP32 rate on this
// part), then FP64.  The column totals wait in shared memory; at the end one
// lane per column runs the p x p solve, so the FP64 solves of a block share
// warp instructions.  Deterministic.
constexpr int BCW = 16, BG = 2 * BCW, BCH = 2 * RED_BOX_ROWS, BMAXC = 128;  // BMAXC: most columns per block
static_assert(BG == RED_BOX_COLS, "one tiled load spans the group's columns");


template <int WS>
struct BulkCfg {
  static constexpr int HB = RED_BOX_ROWS * 4;              // one column's rows in one tiled load: 1 KB
  static constexpr int WB = BCH * WS * 4;                  // the chunk's W32 rows: 8 or 16 KB
  static constexpr int XS = 2 * BG * HB;                   // the group's two tiled loads: 64 KB
  static constexpr int STAGE = XS + WB;                    // 72 or 80 KB
  static constexpr int ST = WS == 4 ? 3 : 2;               // stages
  static constexpr int SMEM = 128 + ST * STAGE + 2 * ST * 8;  // (+ 128: alignment) + the column totals (static)
};

template <int QM, int WS>
__global__ void __launch_bounds__(32 * (BCW + 1), 1) reduce_solve_bulk_kernel(
    const float* __restrict__ Xt, int64_t ldt, int rows, const float* __restrict__ W32,
    const SolveConsts* __restrict__ sc, int q, int ncols, double* __restrict__ b, double* __restrict__ se,
    int* __restrict__ status, const int8_t* __restrict__ shift, DevStatus* st,
    const __grid_constant__ CUtensorMap xmap, int t, int64_t bstride) {
  using K = BulkCfg<WS>;
  constexpr int NA = QM + 2, NW4 = WS / 4, BST = K::ST;
  extern __shared__ __align__(128) uint8_t smem_raw[];
  __shared__ double colsum[BMAXC][NA];  // the block's column totals
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + BST * K::STAGE);
  uint64_t* empty = full + BST;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c_begin = (int)((int64_t)blockIdx.x * ncols / gridDim.x);
  const int c_end = (int)((int64_t)(blockIdx.x + 1) * ncols / gridDim.x);
  const int nch = (rows + BCH - 1) / BCH;
  if (threadIdx.x == 0) {
    for (int s = 0; s < BST; ++s) {
      ptx::mbar_init(&full[s], 1);
      ptx::mbar_init(&empty[s], BCW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    ptx::prefetch_tensormap(&xmap);
  }
  __syncthreads();
  if (warp == BCW) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t it = 0;
      for (int g0 = c_begin; g0 < c_end; g0 += BG) {
        for (int t = 0; t < nch; ++t, ++it) {
          const int s = it % BST;
          const uint32_t r = it / BST;
          if (!ptx::mbar_wait(&empty[s], (r & 1) ^ 1, st)) {
            ptx::settle();  // copies already issued land before the block retires
            return;
          }
          const int rt = rows - t * BCH < BCH ? rows - t * BCH : BCH;
          uint8_t* sb = smem + s * K::STAGE;
          // boxes past the last row or column read zeros (and count their bytes)
          ptx::mbar_arrive_expect_tx(&full[s], (uint32_t)(K::XS + rt * WS * 4));
          ptx::tma_load_2d(sb, &xmap, &full[s], t * BCH, g0);
          ptx::tma_load_2d(sb + BG * K::HB, &xmap, &full[s], t * BCH + RED_BOX_ROWS, g0);
          ptx::bulk_load(sb + K::XS, W32 + (int64_t)t * BCH * WS, rt * WS * 4, &full[s]);
        }
      }
    }
    return;
  }
  // ------------------------------------------------------------ consumers
  uint32_t it = 0;
  bool ok = true;
  for (int g0 = c_begin; g0 < c_end && ok; g0 += BG) {
    const int ca = g0 + 2 * warp;  // this warp's columns: ca, ca + 1
    const bool live0 = ca < c_end, live1 = ca + 1 < c_end;
    float ks[2][NA], kc[2][NA];
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int a = 0; a < NA; ++a) ks[u][a] = kc[u][a] = 0.f;
    for (int t = 0; t < nch; ++t, ++it) {
      const int s = it % BST;
      const uint32_t r = it / BST;
      if (!__all_sync(0xffffffffu, ptx::mbar_wait(&full[s], r & 1, st))) {
        ok = false;
        break;
      }
      if (live0) {
        // column c's rows 0..255 of the chunk at c * HB, rows 256..511 at BG * HB + c * HB
        const float* sx0 = reinterpret_cast<const float*>(smem + s * K::STAGE + (2 * warp) * K::HB);
        const float* sx1 = sx0 + RED_BOX_ROWS;
        const float4* sw = reinterpret_cast<const float4*>(smem + s * K::STAGE + K::XS);
        const int rt = rows - t * BCH < BCH ? rows - t * BCH : BCH;
        float p0[NA], p1[NA];
#pragma unroll
        for (int a = 0; a < NA; ++a) p0[a] = p1[a] = 0.f;
        for (int i = 0; i < rt / 128; ++i) {
#pragma unroll
          for (int rr = 0; rr < 4; ++rr) {
            const int row = i * 128 + rr * 32 + lane;
            const int xo = (i >> 1) * (BG * RED_BOX_ROWS) + (i & 1) * 128 + rr * 32 + lane;
            const float x0 = sx0[xo];
            const float x1 = sx1[xo];
#pragma unroll
            for (int v4 = 0; v4 < NW4; ++v4) {
              const float4 w = sw[row * NW4 + v4];
              const float wr[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
              for (int e = 0; e < 4; ++e)
                if (4 * v4 + e <= QM) {
                  p0[4 * v4 + e] = fmaf(x0, wr[e], p0[4 * v4 + e]);
                  p1[4 * v4 + e] = fmaf(x1, wr[e], p1[4 * v4 + e]);
                }
            }
            p0[QM + 1] = fmaf(x0, x0, p0[QM + 1]);
            p1[QM + 1] = fmaf(x1, x1, p1[QM + 1]);
          }
        }
#pragma unroll
        for (int a = 0; a < NA; ++a) {
          float y = p0[a] - kc[0][a];
          float s2 = ks[0][a] + y;
          kc[0][a] = (s2 - ks[0][a]) - y;
          ks[0][a] = s2;
          y = p1[a] - kc[1][a];
          s2 = ks[1][a] + y;
          kc[1][a] = (s2 - ks[1][a]) - y;
          ks[1][a] = s2;
        }
      }
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&empty[s]);
    }
    if (ok) {
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        if (!(u == 0 ? live0 : live1)) continue;
#pragma unroll
        for (int a = 0; a < NA; ++a) {
          float hi = ks[u][a], lo = -kc[u][a];
#pragma unroll
          for (int o = 16; o; o >>= 1)
            ptx::df_add(hi, lo, __shfl_xor_sync(0xffffffffu, hi, o), __shfl_xor_sync(0xffffffffu, lo, o));
          if (lane == 0) colsum[ca + u - c_begin][a] = (double)hi + (double)lo;
        }
      }
    }
  }
  // every consumer warp is done (or gave up); the solves, one lane per column
  if (!ptx::group_and(1, 32 * BCW, ok)) {
    ptx::settle();  // copies already issued land before the block retires
    return;
  }
  for (int j = threadIdx.x; j < c_end - c_begin; j += 32 * BCW) {
    double sum[NA];
#pragma unroll
    for (int a = 0; a < NA; ++a) sum[a] = colsum[j][a];
    const int col = c_begin + j;
    solve_store<QM>(sum, sc, q, col, b, se, status, shift ? (double)shift[col] : 0.0, t, bstride);
  }
}

cudaError_t preload_reduce_solve_f64() {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, reduce_solve_kernel<3>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, reduce_solve_kernel<7>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, reduce_solve_kernel<QMAX>);
  return e;
}

cudaError_t prepare_reduce_solve() {
  cudaError_t e = cudaFuncSetAttribute(reduce_solve_bulk_kernel<3, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       BulkCfg<4>::SMEM);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(reduce_solve_bulk_kernel<7, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              BulkCfg<8>::SMEM);
}

cudaError_t launch_reduce_solve(const void* Xt, XtKind kind, int64_t ldt, int rows, const double* W,
                                int64_t ldw, const SolveConsts* sc, int q, int ncols, double* b, double* se,
                                int* status, cudaStream_t s, const float* W32, const int8_t* shift,
                                DevStatus* st, int num_sms, const CUtensorMap* xmap, int t, int64_t bstride) {
  if (ncols <= 0) return cudaSuccess;
  if (t < 1 || q + t > QMAX + 1) return cudaErrorInvalidValue;
  if (bstride == 0) bstride = (int64_t)(q + 1) * ncols;
  const int qe = q + t - 1;  // the kernels' bound on the columns of W past the first
  const int grid = (ncols + 7) / 8;
  if (kind == XT_F64) {
    const double* X = static_cast<const double*>(Xt);
    if (qe <= 3)
      reduce_solve_kernel<3><<<grid, 256, 0, s>>>(X, ldt, rows, W, ldw, sc, q, ncols, b, se, status, t, bstride);
    else if (qe <= 7)
      reduce_solve_kernel<7><<<grid, 256, 0, s>>>(X, ldt, rows, W, ldw, sc, q, ncols, b, se, status, t, bstride);
    else
      reduce_solve_kernel<QMAX><<<grid, 256, 0, s>>>(X, ldt, rows, W, ldw, sc, q, ncols, b, se, status, t, bstride);
    return cudaGetLastError();
  }
  if (!W32) return cudaErrorInvalidValue;
  const float* X = static_cast<const float*>(Xt);
  if ((rows % RS_RUN) || (ldt % RS_RUN)) return cudaErrorInvalidValue;  // whole 128-byte runs
  const int g32 = (ncols + 31) / 32;
  const int gb = ncols < num_sms ? ncols : num_sms;  // persistent blocks of the bulk-fed kernel
  const bool bulk = xmap && st && num_sms > 0 && rows % 128 == 0 && (ncols + gb - 1) / gb <= BMAXC;
  if (bulk && qe <= 3)
    reduce_solve_bulk_kernel<3, 4><<<gb, 32 * (BCW + 1), BulkCfg<4>::SMEM, s>>>(X, ldt, rows, W32, sc, q, ncols, b,
                                                                             se, status, shift, st, *xmap, t,
                                                                             bstride);
  else if (bulk && qe <= 7)
    reduce_solve_bulk_kernel<7, 8><<<gb, 32 * (BCW + 1), BulkCfg<8>::SMEM, s>>>(X, ldt, rows, W32, sc, q, ncols, b,
                                                                             se, status, shift, st, *xmap, t,
                                                                             bstride);
  else if (qe <= 3)
    reduce_solve_f32_kernel<3, 4, 16><<<g32, 512, 0, s>>>(X, ldt, rows, W32, sc, q, ncols, b, se, status, shift, t,
                                                          bstride);
  else if (qe <= 7)
    reduce_solve_f32_kernel<7, 8, 16><<<g32, 512, 0, s>>>(X, ldt, rows, W32, sc, q, ncols, b, se, status, shift, t,
                                                          bstride);
  else
    reduce_solve_f32_kernel<QMAX, 16, 8><<<g32, 256, 0, s>>>(X, ldt, rows, W32, sc, q, ncols, b, se, status, shift,
                                                             t, bstride);
  return cudaGetLastError();
}

// The second half of the sums formed by the inverse form's epilogue: per SNP
// column, the total of the 32-row FP32 partials over all row groups, then the
// p x p solve.  A block takes 16 columns (64-byte plane rows) in 32 slices of
// row groups, four groups in flight per thread; every sum is a double-FP32
// pair (B300's FP64 pipe is too narrow for a few million FP64 adds per block):
// each slice over its groups, then the slices pairwise in a fixed tree, so
// the result does not depend on scheduling.  FP64 from the column totals on.
constexpr int PS_COLS = 16, PS_SLICES = 32;

template <int QM>
__global__ void __launch_bounds__(PS_COLS * PS_SLICES)
    partials_solve_kernel(const float* __restrict__ red, int ngroups, int nw, int64_t ldr,
                          const SolveConsts* __restrict__ sc, int q, int ncols, double* __restrict__ b,
                          double* __restrict__ se, int* __restrict__ status, const int8_t* __restrict__ shift, int t,
                          int64_t bstride) {
  __shared__ float2 part[PS_SLICES][QM + 2][PS_COLS];
  __shared__ SolveConsts scs;  // the solves' constants next to the solving threads
  const int cl = threadIdx.x % PS_COLS, slice = threadIdx.x / PS_COLS;
  const int col = blockIdx.x * PS_COLS + cl;
  const int64_t group = (int64_t)(nw + 1) * ldr;
  // every global load is issued before the first use of any (one round trip):
  // this thread's share of the constants (set at init: read before the solve
  // kernel this one depends on has finished), then the SNP's shift and its
  // partials
  constexpr int NW = (int)(sizeof(SolveConsts) / 4), NT = PS_COLS * PS_SLICES, SCW = (NW + NT - 1) / NT;
  int scw[SCW];
#pragma unroll
  for (int j = 0; j < SCW; ++j) {
    const int i = (int)threadIdx.x + j * NT;
    scw[j] = i < NW ? __ldg(reinterpret_cast<const int*>(sc) + i) : 0;
  }
  ptx::griddep_wait();  // a programmatic dependent of the solve kernel that wrote the partials
  const double cshift = (slice == 0 && col < ncols && shift) ? (double)shift[col] : 0.0;
  float hi[QM + 2], lo[QM + 2];
#pragma unroll
  for (int a = 0; a < QM + 2; ++a) hi[a] = lo[a] = 0.f;
  if (col < ncols) {
#pragma unroll 4
    for (int g = slice; g < ngroups; g += PS_SLICES) {
      const float* r = red + g * group + col;
      float v[QM + 2];
#pragma unroll
      for (int a = 0; a <= QM; ++a) v[a] = a < nw ? __ldcs(r + a * ldr) : 0.f;  // W's columns: X~_L, then Y~
      v[QM + 1] = __ldcs(r + nw * ldr);                                         // x~ . x~
#pragma unroll
      for (int a = 0; a < QM + 2; ++a) ptx::df_add(hi[a], lo[a], v[a], 0.f);
    }
  }
#pragma unroll
  for (int a = 0; a < QM + 2; ++a) part[slice][a][cl] = make_float2(hi[a], lo[a]);
#pragma unroll
  for (int j = 0; j < SCW; ++j) {
    const int i = (int)threadIdx.x + j * NT;
    if (i < NW) reinterpret_cast<int*>(&scs)[i] = scw[j];
  }
  for (int w = PS_SLICES / 2; w >= 1; w >>= 1) {  // the first barrier also publishes scs
    __syncthreads();
    if (slice < w) {
#pragma unroll
      for (int a = 0; a < QM + 2; ++a) {
        const float2 o = part[slice + w][a][cl];
        ptx::df_add(hi[a], lo[a], o.x, o.y);
        part[slice][a][cl] = make_float2(hi[a], lo[a]);
      }
    }
  }
  if (slice != 0 || col >= ncols) return;
  double acc[QM + 2];
#pragma unroll
  for (int a = 0; a < QM + 2; ++a) acc[a] = (double)hi[a] + (double)lo[a];
  solve_store<QM>(acc, &scs, q, col, b, se, status, cshift, t, bstride);
}

cudaError_t launch_partials_solve(const float* red, int ngroups, int64_t ldr, const SolveConsts* sc, int q, int t,
                                  int ncols, double* b, double* se, int* status, const int8_t* shift,
                                  cudaStream_t s, int64_t bstride) {
  if (ncols <= 0) return cudaSuccess;
  const int nw = q + t;
  if (t < 1 || nw > 8) return cudaErrorInvalidValue;
  if (bstride == 0) bstride = (int64_t)(q + 1) * ncols;
  // launched as a programmatic dependent of the solve kernel: its blocks start
  // as the solve's CTAs retire and wait (griddep_wait) for all of its stores
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((ncols + PS_COLS - 1) / PS_COLS);
  cfg.blockDim = dim3(PS_COLS * PS_SLICES);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = nw <= 4 ? cudaLaunchKernelEx(&cfg, partials_solve_kernel<3>, red, ngroups, nw, ldr, sc, q, ncols, b,
                                               se, status, shift, t, bstride)
                          : cudaLaunchKernelEx(&cfg, partials_solve_kernel<7>, red, ngroups, nw, ldr, sc, q, ncols, b,
                                               se, status, shift, t, bstride);
  return e != cudaSuccess ? e : cudaGetLastError();
}

// ------------------------------------------- sliced solve: sums from exact products
// The per-SNP inputs of the solve as products of x' (the shifted int8 column)
// with fixed FP64 data (W = M^-1, W^ = [X^_L | Y^] = W [X_L | Y]):
//     S_BL = x~^T X~_L = x'^T X^_L,   r_B = x~^T y~ = x'^T y^,   S_BR = x~^T x~ = x'^T W x' = 2 x'^T T x',
// T = W's lower triangle with its diagonal halved.  C holds, per SNP, the
// exact int32 products of x' with SOLVE_SL slabs of B-bit slices (B =
// SLICED_BITS): slab k row r (r < n_pad) = slice k of (T x')_r in units of
// 2^-Bk / s_T; rows n_pad + e and n_pad + ne + e of slabs 0..2 = slices k and
// k + 3 of W^[:, e]^T x'.  sum_r x'_r C_k[r] is exact in int64 (|x'_r C| <
// 2^39): the product kernel added it over the rows below r_lo into
// acc[k][col]; the rows r_lo .. n - 1 (stored in C) are added here.  The slabs
// and the six slices are then combined in FP64 (smallest first, every factor a
// power of two), then the FP64 solve.
constexpr int SOLVE_SL = SLICED_SLABS;
constexpr double SL_UP = (double)(1 << SLICED_BITS);  // 2^B

template <int QM>
__global__ void __launch_bounds__(256) sliced_solve_kernel(
    const int32_t* __restrict__ C, int64_t ldc, int RS, const long long* __restrict__ fused, int ldacc, int r_lo,
    const __half* __restrict__ xc, int64_t ldx, int n, int n_pad, int ne, const double* __restrict__ inv_scale, const SolveConsts* __restrict__ sc, int q, int t, int ncols,
    double* __restrict__ b, double* __restrict__ se, int* __restrict__ status, const int8_t* __restrict__ shift,
    int64_t bstride) {
  const int lane = threadIdx.x & 31;
  const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (col >= ncols) return;
  const int32_t* cc = C + (int64_t)col * ldc;
  const __half* x = xc + (int64_t)col * ldx;
  long long pk[SOLVE_SL];
#pragma unroll
  for (int k = 0; k < SOLVE_SL; ++k) pk[k] = lane == 0 ? fused[(int64_t)k * ldacc + col] : 0;
#pragma unroll 4
  for (int r = r_lo + lane; r < n; r += 32) {
    const int xi = __half2int_rn(x[r]);
#pragma unroll
    for (int k = 0; k < SOLVE_SL; ++k) pk[k] += (long long)xi * __ldcs(cc + k * RS + r);
  }
#pragma unroll
  for (int k = 0; k < SOLVE_SL; ++k)
#pragma unroll
    for (int o = 16; o; o >>= 1) pk[k] += __shfl_xor_sync(0xffffffffu, pk[k], o);
  // appended row `lane` (< ne): six slices, the smallest first; slice k sits
  // in slab k % 3, row r0 (k < 3) or r1 (k >= 3)
  double ev = 0.0;
  if (lane < ne) {
    const int r0 = n_pad + lane, r1 = n_pad + ne + lane;
    double v = 0.0, f = 1.0 / (SL_UP * SL_UP * SL_UP * SL_UP * SL_UP);  // 2^-5B
#pragma unroll
    for (int k = 5; k >= 1; --k, f *= SL_UP) v = fma((double)cc[(k % 3) * RS + (k < 3 ? r0 : r1)], f, v);
    ev = ((double)cc[r0] + v) * inv_scale[1 + lane];
  }
  double acc[QM + 2];
#pragma unroll
  for (int a = 0; a <= QM; ++a) acc[a] = __shfl_sync(0xffffffffu, ev, a);
  if (lane != 0) return;
  double v = 0.0, f = 1.0;  // |pk| < 2^53: exact conversions
#pragma unroll
  for (int k = 1; k < SOLVE_SL; ++k) f /= SL_UP;  // 2^-B(SOLVE_SL - 1)
#pragma unroll
  for (int k = SOLVE_SL - 1; k >= 1; --k, f *= SL_UP) v = fma((double)pk[k], f, v);
  acc[QM + 1] = 2.0 * ((double)pk[0] + v) * inv_scale[0];
  solve_store<QM>(acc, sc, q, col, b, se, status, shift ? (double)shift[col] : 0.0, t, bstride);
}

cudaError_t launch_sliced_solve(const int32_t* C, int64_t ldc, int RS, const long long* acc, int ldacc, int r_lo,
                                const __half* xc, int64_t ldx, int n, int ne, const double* inv_scale, const SolveConsts* sc, int q, int t, int ncols,
                                double* b, double* se, int* status, const int8_t* shift, cudaStream_t s,
                                int64_t bstride) {
  if (ncols <= 0) return cudaSuccess;
  if (t < 1 || ne != q + t || ne > QMAX + 1) return cudaErrorInvalidValue;
  if (bstride == 0) bstride = (int64_t)(q + 1) * ncols;
  const int n_pad = (int)ldx;
  const int grid = (ncols + 7) / 8;
  if (ne <= 4)
    sliced_solve_kernel<3><<<grid, 256, 0, s>>>(C, ldc, RS, acc, ldacc, r_lo, xc, ldx, n, n_pad, ne, inv_scale, sc, q, t, ncols, b, se,
                                                status, shift, bstride);
  else if (ne <= 8)
    sliced_solve_kernel<7><<<grid, 256, 0, s>>>(C, ldc, RS, acc, ldacc, r_lo, xc, ldx, n, n_pad, ne, inv_scale, sc, q, t, ncols, b, se,
                                                status, shift, bstride);
  else
    sliced_solve_kernel<QMAX><<<grid, 256, 0, s>>>(C, ldc, RS, acc, ldacc, r_lo, xc, ldx, n, n_pad, ne, inv_scale, sc, q, t, ncols, b,
                                                   se, status, shift, bstride);
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
