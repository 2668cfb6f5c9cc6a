// a6, FP64 mode: the blocked triangular solve X~ = L^-1 X over a block of SNP
// columns (Sec. 2.2: packing SNP columns turns trsv into trsm; Sec. 3: the
// trsm is the bottleneck).
//
// With the block operator Aop (row panel k = [-D_k^-1 L_k0 ... | D_k^-1]) the
// output tile (k, c) -- rows k*TB.., SNP columns c*F64_TN.. -- is
//     X~_kc = D_k^-1 X_kc + sum_{j<k} (-D_k^-1 L_kj) X~_jc .
// Tiles of one column strip form a chain in k; strips are independent.  One
// persistent launch hands out tiles in (k, c) order from an atomic counter;
// a tile first applies D_k^-1 to its own (int8 or FP64) input, which needs
// nothing else, then walks j = 0..k-1, waiting on the finished-flag of tile
// (j, c) before reading X~_jc.  A tile only waits on tiles handed out before
// it, and those belong to running CTAs, so the launch cannot deadlock even
// when not all CTAs are resident.  Every wait is bounded (WAIT_LIMIT_NS):
// on expiry the kernel records DEV_ERR_TIMEOUT, raises `abort`, and all CTAs
// return.
#include "gwas_internal.cuh"

namespace gwas {

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ long long globaltimer() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Thread 0 waits until *flag != 0.  Returns false when the launch is aborting.
__device__ bool wait_flag(const int* flag, DevStatus* st) {
  if (ld_acquire(flag) != 0) return true;
  const long long t0 = globaltimer();
  while (true) {
    __nanosleep(200);
    if (ld_acquire(flag) != 0) return true;
    if (*(volatile int*)&st->abort) return false;
    if (globaltimer() - t0 > WAIT_LIMIT_NS) {
      atomicCAS(&st->err, DEV_OK, DEV_ERR_TIMEOUT);
      atomicExch(&st->abort, 1);
      return false;
    }
  }
}

constexpr int KC = 16;  // reduction chunk

// UPPER: the transpose solve X^ = L^-T X with the transpose block operator
// (row panel k = [D_k^-T at block k | -D_k^-T L_jk^T for j > k]); tiles are
// handed out from the last row panel up and tile (k, c) walks j = P-1 .. k+1.
// With identity columns (tri_col0 >= 0, lower) tile (k, c) walks j = jmin ..
// k-1 only, jmin the panel of the strip's first column; tiles k < jmin are zero.
template <typename TIn, bool UPPER>
__global__ void __launch_bounds__(256, 2) trsm_f64_kernel(TrsmF64Args a) {
  __shared__ double As[KC][TB + 1];
  __shared__ double Bs[KC][F64_TN + 1];
  __shared__ int s_tile;
  __shared__ int s_ok;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const TIn* X = static_cast<const TIn*>(a.X);
  int* flags = sched_flags(a.sched);
  const int ntiles = a.P * a.C;

  while (true) {
    if (tid == 0) {
      int t = (int)atomicAdd(&a.sched->counter, 1u);
      if (*(volatile int*)&a.st->abort) t = ntiles;
      s_tile = t;
    }
    __syncthreads();
    const int tile = s_tile;
    if (tile >= ntiles) return;
    const int k = UPPER ? a.P - 1 - tile / a.C : tile / a.C, c = tile % a.C;
    const int col0 = c * F64_TN;
    // identity columns: panels above the strip's first column are zero
    const int jmin = (!UPPER && a.tri_col0 >= 0) ? (int)((a.tri_col0 + col0) / TB) : 0;
    if (k < jmin) {  // a zero tile: stored and published without the solve
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int col = col0 + tx + 16 * q;
        if (col < a.ncols) {
#pragma unroll
          for (int r = 0; r < 8; ++r) a.Xt[(int64_t)col * a.ldt + k * TB + ty + 16 * r] = 0.0;
        }
      }
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        st_release(&flags[k * a.C + c], 1);
      }
      continue;
    }
    const int nsteps = UPPER ? a.P - k : k + 1 - jmin;

    double acc[8][4];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[r][q] = 0.0;

    // j = k first (the diagonal inverse on this tile's own input), then the
    // finished panels, oldest first: 0..k-1 (lower) or P-1..k+1 (upper)
    for (int step = 0; step < nsteps; ++step) {
      const int j = (step == 0) ? k : (UPPER ? a.P - step : jmin + step - 1);
      if (j != k) {
        if (tid == 0) s_ok = wait_flag(&flags[j * a.C + c], a.st) ? 1 : 0;
        __syncthreads();
        if (!s_ok) return;
      }
      const double* Arow = a.Aop + (int64_t)k * TB * a.lda + (int64_t)j * TB;
      for (int t0 = 0; t0 < TB; t0 += KC) {
        // A chunk: rows k*TB + 0..127, reduction index j*TB + t0 .. +15 (row-major, contiguous)
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int e = tid + 256 * r;
          const int row = e / KC, tt = e % KC;
          As[tt][row] = Arow[(int64_t)row * a.lda + t0 + tt];
        }
        // B chunk: rows j*TB + t0 .. +15 of SNP columns col0 .. col0 + 63
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int e = tid + 256 * r;
          const int cc = e / KC, tt = e % KC;
          const int col = col0 + cc;
          const int row = j * TB + t0 + tt;
          double v = 0.0;
          if (col < a.ncols) {
            if (j == k) {
              if (row < a.n) v = (double)X[(int64_t)col * a.ldx + row];
            } else {
              v = __ldcg(&a.Xt[(int64_t)col * a.ldt + row]);
            }
          }
          Bs[tt][cc] = v;
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < KC; ++t) {
          double av[8], bv[4];
#pragma unroll
          for (int r = 0; r < 8; ++r) av[r] = As[t][ty + 16 * r];
#pragma unroll
          for (int q = 0; q < 4; ++q) bv[q] = Bs[t][tx + 16 * q];
#pragma unroll
          for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[r][q] = fma(av[r], bv[q], acc[r][q]);
        }
        __syncthreads();
      }
    }

    // epilogue: X~_kc to global, then publish the tile
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int col = col0 + tx + 16 * q;
      if (col < a.ncols) {
#pragma unroll
        for (int r = 0; r < 8; ++r) a.Xt[(int64_t)col * a.ldt + k * TB + ty + 16 * r] = acc[r][q];
      }
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      st_release(&flags[k * a.C + c], 1);
    }
  }
}

int trsm_f64_grid(int num_sms) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, trsm_f64_kernel<int8_t, false>, 256, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return num_sms * (per_sm < 1 ? 1 : per_sm);
}

cudaError_t preload_trsm_f64_int8() {
  cudaFuncAttributes fa;
  return cudaFuncGetAttributes(&fa, trsm_f64_kernel<int8_t, false>);
}

cudaError_t launch_trsm_f64(const TrsmF64Args& a, bool int8_input, cudaStream_t s, int num_sms, bool upper) {
  if (a.ncols <= 0) return cudaSuccess;
  int per_sm = 0;
  cudaError_t e;
  if (int8_input && upper) return cudaErrorInvalidValue;  // the transpose solve takes FP64 input
  if (int8_input)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, trsm_f64_kernel<int8_t, false>, 256, 0);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, trsm_f64_kernel<double, false>, 256, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int grid = num_sms * per_sm;
  const int ntiles = a.P * a.C;
  if (grid > ntiles) grid = ntiles;
  if (int8_input)
    trsm_f64_kernel<int8_t, false><<<grid, 256, 0, s>>>(a);
  else if (upper)
    trsm_f64_kernel<double, true><<<grid, 256, 0, s>>>(a);
  else
    trsm_f64_kernel<double, false><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace gwas
