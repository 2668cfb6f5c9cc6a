// FP64 set-up kernels: forming M (a1), the blocked Cholesky factorization
// L L^T = M (a2, Sec. 2.1 "potrf M"), the diagonal-block inverses of L (a4)
// and the block operator of the blocked triangular solve.
//
// B300 FP64 runs at a small fraction of the FP32 rate, so these kernels are
// DFMA-bound whatever their memory pattern; they run once per study
// (Sec. 4: set-up is not part of the timed work).
#include <cstdio>

#include "gwas_internal.cuh"

namespace gwas {

// ---------------------------------------------------------------- a1: form M
__global__ void form_m_kernel(const double* __restrict__ phi, int64_t ldphi, int n, int n_pad, double h,
                              double sigma2, int is_L, double* __restrict__ A) {
  const int64_t total = (int64_t)n_pad * n_pad;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n_pad);
    const int j = (int)(e / n_pad);
    double v = 0.0;
    if (i >= j) {
      if (i < n && j < n) {
        const double f = phi[i + j * ldphi];
        v = is_L ? f : sigma2 * (h * f + (i == j ? 1.0 - h : 0.0));
      } else if (i == j) {
        v = 1.0;  // identity on the padding
      }
    }
    A[e] = v;
  }
}

cudaError_t launch_form_m(const double* phi, int64_t ldphi, int n, int n_pad, double h, double sigma2,
                          int is_L, double* A, cudaStream_t s) {
  form_m_kernel<<<1184, 256, 0, s>>>(phi, ldphi, n, n_pad, h, sigma2, is_L, A);
  return cudaGetLastError();
}

// ------------------------------------------------- diagonal block: potrf + trtri
// One CTA factors the TB x TB diagonal block k (already updated by the earlier
// panels), writes L_kk back and writes D_k^-1 = L_kk^-1.  Both triangles are
// held packed column-major in shared memory: entry (i, j), i >= j, at
// j * TB - j * (j - 1) / 2 + (i - j).
__device__ __forceinline__ int pk(int i, int j) { return j * TB - (j * (j - 1)) / 2 + (i - j); }

constexpr int PACKED = TB * (TB + 1) / 2;

// factor = 0: the block already holds L_kk (a caller-supplied factor); only
// its diagonal is checked and its inverse formed.  Block index k = k0 + blockIdx.x.
__global__ void __launch_bounds__(256) potrf_diag_kernel(double* __restrict__ A, int64_t lda, int k0,
                                                         double* __restrict__ Dinv, DevStatus* st, int factor) {
  const int k = k0 + blockIdx.x;
  extern __shared__ double smem[];
  double* Lp = smem;           // packed L_kk
  double* Xp = smem + PACKED;  // packed L_kk^-1
  __shared__ double s_d;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  double* Akk = A + (int64_t)k * TB * lda + (int64_t)k * TB;

  for (int j = warp; j < TB; j += nw)
    for (int i = j + lane; i < TB; i += 32) Lp[pk(i, j)] = Akk[i + j * lda];
  __syncthreads();

  for (int j = 0; j < TB && factor; ++j) {
    if (tid == 0) {
      double d = Lp[pk(j, j)];
      if (!(d > 0.0)) {  // not positive definite (or NaN): record, continue with 1
        atomicMin(&st->not_spd, (unsigned long long)(k * TB + j));
        d = 1.0;
      }
      d = sqrt(d);
      Lp[pk(j, j)] = d;
      s_d = d;
    }
    __syncthreads();
    const double d = s_d;
    for (int i = j + 1 + tid; i < TB; i += blockDim.x) Lp[pk(i, j)] /= d;
    __syncthreads();
    for (int t = j + 1 + warp; t < TB; t += nw) {
      const double ltj = Lp[pk(t, j)];
      for (int i = t + lane; i < TB; i += 32) Lp[pk(i, t)] -= Lp[pk(i, j)] * ltj;
    }
    __syncthreads();
  }

  if (!factor && tid < TB && !(Lp[pk(tid, tid)] > 0.0)) {
    atomicMin(&st->not_spd, (unsigned long long)(k * TB + tid));
    Lp[pk(tid, tid)] = 1.0;
  }
  __syncthreads();
  // L_kk back to A (strict upper triangle of the block zeroed)
  for (int j = warp; j < TB; j += nw)
    for (int i = lane; i < TB; i += 32) Akk[i + j * lda] = (i >= j) ? Lp[pk(i, j)] : 0.0;

  // L_kk^-1, column c by forward substitution of e_c (one thread per column)
  if (tid < TB) {
    const int c = tid;
    Xp[pk(c, c)] = 1.0 / Lp[pk(c, c)];
    for (int i = c + 1; i < TB; ++i) {
      double v = 0.0;
      for (int t = c; t < i; ++t) v += Lp[pk(i, t)] * Xp[pk(t, c)];
      Xp[pk(i, c)] = -v / Lp[pk(i, i)];
    }
  }
  __syncthreads();
  double* D = Dinv + (int64_t)k * TB * TB;
  for (int j = warp; j < TB; j += nw)
    for (int i = lane; i < TB; i += 32) D[i + j * TB] = (i >= j) ? Xp[pk(i, j)] : 0.0;
}

// ---------------------------------------------------------- generic FP64 GEMM
// C(i, j) = alpha * sum_t A(i, t) B(j, t) + beta * C(i, j),  i < M, j < N.
// Element (i, t) of A is at A[i * a_i + t * a_t] (likewise B and C), so any
// transposition is a choice of strides.  lower = 1 skips 64 x 64 output tiles
// strictly above the diagonal (symmetric rank-k updates).
struct DgemmArgs {
  int M, N, K;
  const double* A;
  int64_t a_i, a_t;
  const double* B;
  int64_t b_j, b_t;
  double* C;
  int64_t c_i, c_j;
  double alpha, beta;
  int lower;
};

constexpr int DG_T = 64, DG_K = 16;

__global__ void __launch_bounds__(256) dgemm_kernel(DgemmArgs g) {
  const int ti = blockIdx.y, tj = blockIdx.x;
  if (g.lower && tj > ti) return;
  __shared__ double As[DG_K][DG_T + 1];
  __shared__ double Bs[DG_K][DG_T + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int i0 = ti * DG_T, j0 = tj * DG_T;
  double acc[4][4] = {};
  for (int t0 = 0; t0 < g.K; t0 += DG_K) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = tid + 256 * r;
      int ii, tt;
      if (g.a_i == 1) { ii = e % DG_T; tt = e / DG_T; } else { tt = e % DG_K; ii = e / DG_K; }
      const int gi = i0 + ii, gt = t0 + tt;
      As[tt][ii] = (gi < g.M && gt < g.K) ? g.A[gi * g.a_i + gt * g.a_t] : 0.0;
      int jj, uu;
      if (g.b_j == 1) { jj = e % DG_T; uu = e / DG_T; } else { uu = e % DG_K; jj = e / DG_K; }
      const int gj = j0 + jj, gu = t0 + uu;
      Bs[uu][jj] = (gj < g.N && gu < g.K) ? g.B[gj * g.b_j + gu * g.b_t] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < DG_K; ++t) {
      double a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) { a[r] = As[t][ty + 16 * r]; b[r] = Bs[t][tx + 16 * r]; }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int gi = i0 + ty + 16 * r, gj = j0 + tx + 16 * c;
      if (gi < g.M && gj < g.N) {
        double* cp = g.C + gi * g.c_i + gj * g.c_j;
        *cp = g.alpha * acc[r][c] + (g.beta != 0.0 ? g.beta * *cp : 0.0);
      }
    }
}

static cudaError_t dgemm(const DgemmArgs& g, cudaStream_t s, int64_t* launches) {
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  dim3 grid((g.N + DG_T - 1) / DG_T, (g.M + DG_T - 1) / DG_T);
  dgemm_kernel<<<grid, 256, 0, s>>>(g);
  ++*launches;
  return cudaGetLastError();
}

// ------------------------------------------------ a2: blocked right-looking potrf
cudaError_t launch_potrf(double* A, int n_pad, double* Dinv, double* panel, DevStatus* st, cudaStream_t s,
                         int64_t* launches) {
  const int P = n_pad / TB;
  const size_t smem = 2 * PACKED * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(potrf_diag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t lda = n_pad;
  for (int k = 0; k < P; ++k) {
    potrf_diag_kernel<<<1, 256, smem, s>>>(A, lda, k, Dinv, st, 1);
    ++*launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int rows = n_pad - (k + 1) * TB;
    if (rows == 0) break;
    double* Aik = A + (int64_t)k * TB * lda + (k + 1) * TB;  // rows below, block column k
    // panel = A_ik D_k^-T  (L_ik for all i > k)
    DgemmArgs g{};
    g.M = rows; g.N = TB; g.K = TB;
    g.A = Aik; g.a_i = 1; g.a_t = lda;
    g.B = Dinv + (int64_t)k * TB * TB; g.b_j = 1; g.b_t = TB;  // B(j, t) = Dinv(j, t)
    g.C = panel; g.c_i = 1; g.c_j = n_pad;
    g.alpha = 1.0; g.beta = 0.0; g.lower = 0;
    if ((e = dgemm(g, s, launches)) != cudaSuccess) return e;
    e = cudaMemcpy2DAsync(Aik, lda * sizeof(double), panel, (size_t)n_pad * sizeof(double),
                          rows * sizeof(double), TB, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    // trailing symmetric update A_22 -= L_21 L_21^T (lower tiles only)
    DgemmArgs u{};
    u.M = rows; u.N = rows; u.K = TB;
    u.A = panel; u.a_i = 1; u.a_t = n_pad;
    u.B = panel; u.b_j = 1; u.b_t = n_pad;
    double* A22 = A + (int64_t)(k + 1) * TB * lda + (k + 1) * TB;
    u.C = A22; u.c_i = 1; u.c_j = lda;
    u.alpha = -1.0; u.beta = 1.0; u.lower = 1;
    if ((e = dgemm(u, s, launches)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_invert_diag_blocks(double* L, int n_pad, double* Dinv, DevStatus* st, cudaStream_t s) {
  const size_t smem = 2 * PACKED * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(potrf_diag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  potrf_diag_kernel<<<n_pad / TB, 256, smem, s>>>(L, n_pad, 0, Dinv, st, 0);
  return cudaGetLastError();
}

// ------------------------------------------------------ a4: the block operator
__global__ void put_diag_inverses_kernel(const double* __restrict__ Dinv, int P, int64_t n_pad,
                                         double* __restrict__ Aop) {
  const int k = blockIdx.x;
  const double* D = Dinv + (int64_t)k * TB * TB;
  for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
    const int i = e / TB, j = e % TB;  // row-major destination: consecutive j
    Aop[((int64_t)k * TB + i) * n_pad + (int64_t)k * TB + j] = D[i + j * TB];
  }
}

cudaError_t launch_build_aop(const double* L, const double* Dinv, int n_pad, double* Aop, cudaStream_t s,
                             int64_t* launches) {
  const int P = n_pad / TB;
  cudaError_t e;
  for (int k = 1; k < P; ++k) {
    // Aop[k-panel rows, 0 : k*TB] = -D_k^-1 L[k-panel rows, 0 : k*TB]
    DgemmArgs g{};
    g.M = TB; g.N = k * TB; g.K = TB;
    g.A = Dinv + (int64_t)k * TB * TB; g.a_i = 1; g.a_t = TB;
    g.B = L + (int64_t)k * TB; g.b_j = n_pad; g.b_t = 1;  // B(j, t) = L(k*TB + t, j)
    g.C = Aop + (int64_t)k * TB * n_pad; g.c_i = n_pad; g.c_j = 1;
    g.alpha = -1.0; g.beta = 0.0; g.lower = 0;
    if ((e = dgemm(g, s, launches)) != cudaSuccess) return e;
  }
  put_diag_inverses_kernel<<<P, 256, 0, s>>>(Dinv, P, n_pad, Aop);
  ++*launches;
  return cudaGetLastError();
}

// --------------------------------------------- the transpose block operator
__global__ void put_diag_inverses_t_kernel(const double* __restrict__ Dinv, int P, int64_t n_pad,
                                           double* __restrict__ AopT) {
  const int k = blockIdx.x;
  const double* D = Dinv + (int64_t)k * TB * TB;
  for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
    const int i = e / TB, j = e % TB;  // AopT[k-panel row i][k-block col j] = D_k^-T(i, j) = D_k^-1(j, i)
    AopT[((int64_t)k * TB + i) * n_pad + (int64_t)k * TB + j] = D[j + i * TB];
  }
}

cudaError_t launch_build_aop_t(const double* L, const double* Dinv, int n_pad, double* AopT, cudaStream_t s,
                               int64_t* launches) {
  const int P = n_pad / TB;
  cudaError_t e;
  for (int k = 0; k + 1 < P; ++k) {
    // AopT[k-panel rows, (k+1)TB :] = -D_k^-T L[(k+1)TB :, k-panel cols]^T
    DgemmArgs g{};
    g.M = TB; g.N = n_pad - (k + 1) * TB; g.K = TB;
    g.A = Dinv + (int64_t)k * TB * TB; g.a_i = TB; g.a_t = 1;                // A(i, t) = D_k^-1(t, i)
    g.B = L + (int64_t)k * TB * n_pad + (k + 1) * TB; g.b_j = 1; g.b_t = n_pad;  // B(j, t) = L((k+1)TB + j, kTB + t)
    g.C = AopT + (int64_t)k * TB * n_pad + (k + 1) * TB; g.c_i = n_pad; g.c_j = 1;
    g.alpha = -1.0; g.beta = 0.0; g.lower = 0;
    if ((e = dgemm(g, s, launches)) != cudaSuccess) return e;
  }
  put_diag_inverses_t_kernel<<<P, 256, 0, s>>>(Dinv, P, n_pad, AopT);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace gwas
