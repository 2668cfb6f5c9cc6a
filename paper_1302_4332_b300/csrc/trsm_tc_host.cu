// Host side of the split-precision solve (a4 split copies, a6, a10's batched
// launch): per-study state, set-up (the split block
// operator, the pair form, L^-1 for the inverse form), tensor maps, tile
// orders, and the small set-up and pre-pass kernels.  The solve kernels
// themselves are in trsm_tc.cu.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "tc_ptx.cuh"
#include "trsm_tc_kernels.cuh"

namespace gwas {
namespace tc {

// ------------------------------------------- per-SNP integer shift (pre-pass)
// c_i = round(mean of the n dosages of SNP i), from an exact integer sum.
__global__ void column_shift_kernel(const int8_t* __restrict__ X, int64_t ldx, int n, int ncols,
                                    int8_t* __restrict__ shift) {
  const int lane = threadIdx.x & 31;
  const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (col >= ncols) return;
  const int8_t* x = X + (int64_t)col * ldx;  // 16-byte aligned (checked by the caller)
  int sum = 0;
  const int n16 = n & ~15;
  for (int r = lane * 16; r < n16; r += 32 * 16) {
    const int4 v = __ldg(reinterpret_cast<const int4*>(x + r));
    const int w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) sum += __dp4a(w[i], 0x01010101, 0);
  }
  for (int r = n16 + lane; r < n; r += 32) sum += x[r];
#pragma unroll
  for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if (lane == 0) {
    const long long num = 2LL * sum + n;  // floor((2 sum + n) / 2n) = round-half-up of sum / n
    const long long den = 2LL * n;
    long long c = num >= 0 ? num / den : -((-num + den - 1) / den);
    if (c > 127) c = 127;
    if (c < -127) c = -127;
    shift[col] = (int8_t)c;
  }
}

// 16 consecutive values of the cast block at element offset `off` (a multiple
// of 16): BF16, FP32 (read as TF32) or FP16 -- all exact for |x - c_i| <= 255.
enum CastOut : int { OUT_BF16 = 0, OUT_F32 = 1, OUT_F16 = 2 };
template <int OUT>
__device__ __forceinline__ void store_cast16(void* xc, int64_t off, const float (&f)[16]) {
  if constexpr (OUT == OUT_F32) {
    float4* o = reinterpret_cast<float4*>(static_cast<float*>(xc) + off);
#pragma unroll
    for (int i = 0; i < 4; ++i) o[i] = make_float4(f[4 * i], f[4 * i + 1], f[4 * i + 2], f[4 * i + 3]);
  } else {
    uint32_t wv[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if constexpr (OUT == OUT_F16) {
        const __half2 h2 = __floats2half2_rn(f[2 * i], f[2 * i + 1]);
        wv[i] = *reinterpret_cast<const uint32_t*>(&h2);
      } else {
        const __nv_bfloat162 b2 = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
        wv[i] = *reinterpret_cast<const uint32_t*>(&b2);
      }
    }
    uint4* o = reinterpret_cast<uint4*>(static_cast<uint16_t*>(xc) + off);
    o[0] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
    o[1] = make_uint4(wv[4], wv[5], wv[6], wv[7]);
  }
}

// 16 rows of a 2-bit packed column (4 bytes, row 4k + i in bits 2i .. 2i+1 of
// byte k) as the 16 int8 values of an int4: v_i = the codes of rows 4k + i
// (one per byte k), then a 4 x 4 byte transpose by byte permutes, so that
// word k holds rows 4k .. 4k+3 (13 operations for the 16 values).
__device__ __forceinline__ int4 unpack16(uint32_t p) {
  const uint32_t v0 = p & 0x03030303u, v1 = (p >> 2) & 0x03030303u;
  const uint32_t v2 = (p >> 4) & 0x03030303u, v3 = (p >> 6) & 0x03030303u;
  const uint32_t t0 = __byte_perm(v0, v1, 0x5140), t1 = __byte_perm(v2, v3, 0x5140);  // bytes 0, 1
  const uint32_t t2 = __byte_perm(v0, v1, 0x7362), t3 = __byte_perm(v2, v3, 0x7362);  // bytes 2, 3
  return make_int4((int)__byte_perm(t0, t1, 0x5410), (int)__byte_perm(t0, t1, 0x7632),
                   (int)__byte_perm(t2, t3, 0x5410), (int)__byte_perm(t2, t3, 0x7632));
}

// The same in one read of the column: for n <= 512 * NV each lane holds its
// NV 16-row pieces of the column in registers between the sum and the cast
// (all of them in flight at once).  PK: the column is 2-bit packed (ldx bytes
// per column, ceil(n/4) of them used; 4 bytes a piece), as the packed input
// forms carry hard-called genotypes -- no int8 copy of the block is made.
template <int OUT, int NV, bool PK = false>
__device__ __forceinline__ void cast_column_reg(const int8_t* __restrict__ X, int64_t ldx, int n, int n_pad,
                                                int col, int8_t* __restrict__ shift, void* __restrict__ xc) {
  const int lane = threadIdx.x & 31;
  const int8_t* x = X + (int64_t)col * ldx;  // 16-byte aligned (checked by the caller)
  int4 v[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    const int r = j * 512 + lane * 16;
    if (PK) {
      const int nb = (n + 3) / 4;  // packed bytes of the column; rows past n are 0 in them
      const uint8_t* xb = reinterpret_cast<const uint8_t*>(x) + r / 4;
      uint32_t p = 0;
      if (r + 16 <= n) {
        p = __ldg(reinterpret_cast<const uint32_t*>(xb));
        v[j] = unpack16(p);
      } else {  // the ragged piece: rows past n as 0 whatever their bits hold
        for (int k = 0; r / 4 + k < nb && k < 4; ++k) p |= (uint32_t)xb[k] << (8 * k);
        const int4 q = unpack16(p);
        uint32_t w[4] = {(uint32_t)q.x, (uint32_t)q.y, (uint32_t)q.z, (uint32_t)q.w};
        for (int i = 0; i < 16; ++i)
          if (r + i >= n) w[i >> 2] &= ~(0xFFu << (8 * (i & 3)));
        v[j] = make_int4((int)w[0], (int)w[1], (int)w[2], (int)w[3]);
      }
    } else if (r + 16 <= n) {
      v[j] = __ldg(reinterpret_cast<const int4*>(x + r));
    } else {  // the ragged piece (bytes past n read as 0)
      uint32_t w[4] = {0u, 0u, 0u, 0u};
      for (int i = 0; i < 16 && r + i < n; ++i) w[i >> 2] |= (uint32_t)(uint8_t)x[r + i] << (8 * (i & 3));
      v[j] = make_int4((int)w[0], (int)w[1], (int)w[2], (int)w[3]);
    }
  }
  int c = 0;
  if (shift) {
    int sum = 0;
#pragma unroll
    for (int j = 0; j < NV; ++j)
      sum += __dp4a(v[j].x, 0x01010101, 0) + __dp4a(v[j].y, 0x01010101, 0) + __dp4a(v[j].z, 0x01010101, 0) +
             __dp4a(v[j].w, 0x01010101, 0);
#pragma unroll
    for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    const long long num = 2LL * sum + n, den = 2LL * n;
    long long cc = num >= 0 ? num / den : -((-num + den - 1) / den);
    cc = cc > 127 ? 127 : (cc < -127 ? -127 : cc);
    c = (int)cc;
    if (lane == 0) shift[col] = (int8_t)c;
  }
#pragma unroll
  for (int j = 0; j <= NV; ++j) {  // piece NV: padding rows only (zeros)
    const int r = j * 512 + lane * 16;
    if (r >= n_pad) break;
    float f[16];
    const int w[4] = {j < NV ? v[j].x : 0, j < NV ? v[j].y : 0, j < NV ? v[j].z : 0, j < NV ? v[j].w : 0};
#pragma unroll
    for (int i = 0; i < 16; ++i)
      f[i] = r + i < n ? (float)((int)(int8_t)(w[i >> 2] >> (8 * (i & 3))) - c) : 0.f;
    store_cast16<OUT>(xc, (int64_t)col * n_pad + r, f);
  }
}

// Launch order of a block (inverse form): this cast (an ordinary launch: its
// input may come from any kernel before it), then the solve as its
// programmatic dependent, then the sums' kernel as the solve's.  The cast
// zeroes the solve's unit counter (no stream operation between it and the
// solve) and writes the cast block and this block's shift slot.
template <int OUT, int NV, bool PK = false>
__global__ void __launch_bounds__(256) cast_shift_reg_kernel(const int8_t* __restrict__ X, int64_t ldx, int n,
                                                             int n_pad, int ncols, int8_t* __restrict__ shift,
                                                             void* __restrict__ xc, unsigned int* counter) {
  ptx::griddep_launch();  // the solve kernel may start its set-up
  if (counter && blockIdx.x == 0 && threadIdx.x == 0) *counter = 0;
  const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (col < ncols) cast_column_reg<OUT, NV, PK>(X, ldx, n, n_pad, col, shift, xc);
}

// B operand of the inverse form: x'_ri = x_ri - c_i on rows < n and 0 on rows
// n..n_pad-1, as BF16, FP32 (read as TF32 by the tensor cores) or FP16,
// column-major with leading dimension n_pad.  c_i is computed here as in
// column_shift_kernel when `shift` is given (and stored there), else 0.  One
// warp per SNP column.
template <int OUT>
__device__ __forceinline__ void cast_column(const int8_t* __restrict__ X, int64_t ldx, int n, int n_pad, int col,
                                            int8_t* __restrict__ shift, void* __restrict__ xc) {
  const int lane = threadIdx.x & 31;
  const int8_t* x = X + (int64_t)col * ldx;  // 16-byte aligned (checked by the caller)
  const int n16 = n & ~15;
  int c = 0;
  if (shift) {
    int sum = 0;
    int r = lane * 16;
    for (; r + 3 * 512 < n16; r += 4 * 512) {  // four independent 16-byte loads in flight per lane
      int4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = __ldg(reinterpret_cast<const int4*>(x + r + u * 512));
#pragma unroll
      for (int u = 0; u < 4; ++u)
        sum += __dp4a(v[u].x, 0x01010101, 0) + __dp4a(v[u].y, 0x01010101, 0) + __dp4a(v[u].z, 0x01010101, 0) +
               __dp4a(v[u].w, 0x01010101, 0);
    }
    for (; r < n16; r += 512) {
      const int4 v = __ldg(reinterpret_cast<const int4*>(x + r));
      sum += __dp4a(v.x, 0x01010101, 0) + __dp4a(v.y, 0x01010101, 0) + __dp4a(v.z, 0x01010101, 0) +
             __dp4a(v.w, 0x01010101, 0);
    }
    for (int r2 = n16 + lane; r2 < n; r2 += 32) sum += x[r2];
#pragma unroll
    for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    const long long num = 2LL * sum + n, den = 2LL * n;
    long long cc = num >= 0 ? num / den : -((-num + den - 1) / den);
    cc = cc > 127 ? 127 : (cc < -127 ? -127 : cc);
    c = (int)cc;
    if (lane == 0) shift[col] = (int8_t)c;
  }
#pragma unroll 2
  for (int r = lane * 16; r < n_pad; r += 32 * 16) {  // n_pad is a multiple of 128
    float f[16];
    if (r + 16 <= n) {
      const int4 v = __ldg(reinterpret_cast<const int4*>(x + r));
      const int w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int i = 0; i < 16; ++i) f[i] = (float)((int)(int8_t)(w[i >> 2] >> (8 * (i & 3))) - c);
    } else {
#pragma unroll
      for (int i = 0; i < 16; ++i) f[i] = (r + i < n) ? (float)((int)x[r + i] - c) : 0.f;
    }
    store_cast16<OUT>(xc, (int64_t)col * n_pad + r, f);
  }
}

template <int OUT>
__global__ void cast_shift_kernel(const int8_t* __restrict__ X, int64_t ldx, int n, int n_pad, int ncols,
                                  int8_t* __restrict__ shift, void* __restrict__ xc, unsigned int* counter) {
  ptx::griddep_launch();  // the solve kernel may start its set-up
  if (counter && blockIdx.x == 0 && threadIdx.x == 0) *counter = 0;
  const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (col < ncols) cast_column<OUT>(X, ldx, n, n_pad, col, shift, xc);
}

// The cast pre-pass of the inverse form: one read per column while it fits
// the registers (n <= 16384), else two.  counter: the solve's unit counter to
// zero, or null when the caller clears it.
template <int OUT>
static cudaError_t launch_cast_t(const int8_t* X, int64_t ldx, int n, int n_pad, int ncols, int8_t* shift, void* xc,
                                 unsigned int* counter, cudaStream_t s, bool packed = false) {
  const int grid = (ncols + 7) / 8;
  if (packed) {  // 2-bit packed columns: the register form only
    if (n <= 512 * 20)
      cast_shift_reg_kernel<OUT, 20, true><<<grid, 256, 0, s>>>(X, ldx, n, n_pad, ncols, shift, xc, counter);
    else if (n <= 512 * 32)
      cast_shift_reg_kernel<OUT, 32, true><<<grid, 256, 0, s>>>(X, ldx, n, n_pad, ncols, shift, xc, counter);
    else
      return cudaErrorInvalidValue;
    return cudaGetLastError();
  }
  if (n <= 512 * 20)
    cast_shift_reg_kernel<OUT, 20><<<grid, 256, 0, s>>>(X, ldx, n, n_pad, ncols, shift, xc, counter);
  else if (n <= 512 * 32)
    cast_shift_reg_kernel<OUT, 32><<<grid, 256, 0, s>>>(X, ldx, n, n_pad, ncols, shift, xc, counter);
  else
    cast_shift_kernel<OUT><<<grid, 256, 0, s>>>(X, ldx, n, n_pad, ncols, shift, xc, counter);
  return cudaGetLastError();
}

static cudaError_t launch_cast(int out, const int8_t* X, int64_t ldx, int n, int n_pad, int ncols, int8_t* shift,
                               void* xc, unsigned int* counter, cudaStream_t s, bool packed = false) {
  if (out == OUT_F32) return launch_cast_t<OUT_F32>(X, ldx, n, n_pad, ncols, shift, xc, counter, s, packed);
  if (out == OUT_F16) return launch_cast_t<OUT_F16>(X, ldx, n, n_pad, ncols, shift, xc, counter, s, packed);
  return launch_cast_t<OUT_BF16>(X, ldx, n, n_pad, ncols, shift, xc, counter, s, packed);
}

// The batch's cast pre-passes in one launch: the columns of every study of a
// step, one warp per column (the study found from its first column), each
// cast as cast_shift_reg_kernel casts it; the batch's unit counter zeroed.
// One launch instead of a memset and a cast per study keeps the gaps between
// graph nodes out of the step, and the solve follows as its programmatic
// dependent.
struct CastJob {
  const int8_t* X;
  int64_t ldx;
  int n, n_pad, col0, ncols;
  int8_t* shift;
  void* xc;
};
struct CastJobs {
  CastJob j[MAX_STUDIES];
  int njobs, total;
  unsigned int* counter;
};

template <int OUT, int NV>
__global__ void __launch_bounds__(256) cast_batch_kernel(const __grid_constant__ CastJobs J) {
  ptx::griddep_launch();  // the solve kernel may start its set-up
  if (blockIdx.x == 0 && threadIdx.x == 0) *J.counter = 0;
  const int g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (g >= J.total) return;
  int i = 0;
  while (i + 1 < J.njobs && g >= J.j[i + 1].col0) ++i;
  const CastJob& c = J.j[i];
  cast_column_reg<OUT, NV>(c.X, c.ldx, c.n, c.n_pad, g - c.col0, c.shift, c.xc);
}

template <int OUT>
static cudaError_t launch_cast_batch_t(const CastJobs& J, int nmax, cudaStream_t s) {
  const int grid = (J.total + 7) / 8;
  if (nmax <= 512 * 20)
    cast_batch_kernel<OUT, 20><<<grid, 256, 0, s>>>(J);
  else
    cast_batch_kernel<OUT, 32><<<grid, 256, 0, s>>>(J);
  return cudaGetLastError();
}

// Columns c0.. c0+ncols-1 of the n_pad x n_pad identity as int8, column-major
// with leading dimension n_pad (the right-hand side that turns the
// substitution into L^-1).
__global__ void identity_i8_kernel(int8_t* __restrict__ I8, int n_pad, int c0, int ncols) {
  const int64_t total = (int64_t)n_pad * ncols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int col = (int)(e / n_pad), row = (int)(e % n_pad);
    I8[e] = row == c0 + col ? 1 : 0;
  }
}

// Columns c0.. of L^-1, solved in FP64 into `xt` (column-major, leading
// dimension ldt), transposed into the row-major hi/lo pieces of the inverse
// form's operator: hi = v rounded to BF16 / TF32, lo = (v - hi) rounded, both
// from the FP64 value.  Entries above the diagonal and in the padding rows and
// columns (index >= n) are set to zero.  32 x 32 tiles through shared memory.
template <bool TF32>
__global__ void linv_split_kernel(const double* __restrict__ xt, int64_t ldt, int n, int n_pad, int c0, int ncols,
                                  void* __restrict__ hi, void* __restrict__ lo) {
  __shared__ double tile[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  const int q0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int q = q0 + ty + 8 * i;
    tile[ty + 8 * i][tx] = q < ncols ? xt[(int64_t)q * ldt + r0 + tx] : 0.0;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int row = r0 + ty + 8 * i, q = q0 + tx, gcol = c0 + q;
    if (q >= ncols) continue;
    double v = tile[tx][ty + 8 * i];
    if (row >= n || gcol >= n || gcol > row) v = 0.0;
    const int64_t idx = (int64_t)row * n_pad + gcol;
    if constexpr (TF32) {
      uint32_t hb;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hb) : "f"((float)v));
      const float h = __uint_as_float(hb);
      static_cast<float*>(hi)[idx] = h;
      static_cast<float*>(lo)[idx] = (float)(v - (double)h);
    } else {
      const __nv_bfloat16 h = __float2bfloat16_rn((float)v);
      static_cast<__nv_bfloat16*>(hi)[idx] = h;
      static_cast<__nv_bfloat16*>(lo)[idx] = __float2bfloat16_rn((float)(v - (double)__bfloat162float(h)));
    }
  }
}

// FP16 form of the inverse's pieces.  linv_rows_kernel transposes solved
// columns of L^-1 into a row-major FP32 copy (upper triangle and padding
// zeroed, as linv_split_kernel); then per row r, with m_r = max_j |L^-1_rj|,
// the row is scaled by s_r = 2^(14 - e_r), 2^(e_r - 1) <= m_r < 2^e_r (so
// |s_r L^-1_rj| < 2^15, inside FP16's range with 11 significant bits for the
// hi piece and 11 more for the lo piece, both exact FP32 operations), and
// rscale[r] = 1 / s_r.
__global__ void linv_rows_kernel(const double* __restrict__ xt, int64_t ldt, int n, int n_pad, int c0, int ncols,
                                 double* __restrict__ rows64) {
  __shared__ double tile[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  const int q0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int q = q0 + ty + 8 * i;
    tile[ty + 8 * i][tx] = q < ncols ? xt[(int64_t)q * ldt + r0 + tx] : 0.0;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int row = r0 + ty + 8 * i, q = q0 + tx, gcol = c0 + q;
    if (q >= ncols) continue;
    double v = tile[tx][ty + 8 * i];
    if (row >= n || gcol >= n || gcol > row) v = 0.0;
    rows64[(int64_t)row * n_pad + gcol] = v;
  }
}

// One block per row of L^-1: its scale, then its FP16 hi/lo pieces.
__global__ void __launch_bounds__(256) linv_split_f16_kernel(const double* __restrict__ rows64, int n_pad,
                                                             __half* __restrict__ hi, __half* __restrict__ lo,
                                                             float* __restrict__ rscale) {
  __shared__ float wmax[8];
  const int row = blockIdx.x;
  const double* src = rows64 + (int64_t)row * n_pad;
  float m = 0.f;
  for (int j = threadIdx.x; j <= row && j < n_pad; j += 256) m = fmaxf(m, (float)fabs(src[j]));
#pragma unroll
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
  __syncthreads();
  m = wmax[0];
#pragma unroll
  for (int w = 1; w < 8; ++w) m = fmaxf(m, wmax[w]);
  int e = 0;
  if (m > 0.f) frexpf(m, &e);  // m = f * 2^e, 0.5 <= f < 1
  const float sc = ldexpf(1.f, 14 - e);
  if (threadIdx.x == 0) rscale[row] = ldexpf(1.f, e - 14);
  for (int j = threadIdx.x; j < n_pad; j += 256) {
    const double v = src[j] * (double)sc;  // a power of two: exact
    const __half h = __float2half_rn((float)v);
    hi[(int64_t)row * n_pad + j] = h;
    lo[(int64_t)row * n_pad + j] = __float2half_rn((float)(v - (double)__half2float(h)));
  }
}

// ------------------------------------------------------------ set-up kernels
// Pair form of the block operator (FP64, set-up of the pair product): the odd
// row panels re-expressed through the even one before them, so neither row of
// a pair needs the other's result.  With A = Aop (row panel k =
// [A_k0 .. A_k,k-1 | A_kk = D_k^-1], row-major, leading dimension ld) and a
// pair (2u, 2u+1):
//   A'_{2u+1,j}  = A_{2u+1,j} + A_{2u+1,2u} A_{2u,j}   (j < 2u)
//   A'_{2u+1,2u} = A_{2u+1,2u} A_{2u,2u}               (it multiplies the int8 X_{2u})
// (A'_{2u+1,2u+1} = A_{2u+1,2u+1}), from substituting panel 2u's equation
// X~_{2u} = sum_{j<2u} A_{2u,j} X~_j + A_{2u,2u} X_{2u} into panel 2u+1's.
// `out` holds a copy of Aop; this kernel overwrites the odd rows' columns
// < (2u+1)*TB.  Block (x, u): rows of panel 2u+1, columns 64x .. 64x+63.
__global__ void __launch_bounds__(256) pair_rows_kernel(const double* __restrict__ A, double* __restrict__ out,
                                                        int64_t ld, int P) {
  const int k0 = 2 * blockIdx.y, k1 = k0 + 1;
  const int c0 = blockIdx.x * 64;
  if (k1 >= P || c0 >= k1 * TB) return;
  constexpr int KC = 16;             // t per chunk
  __shared__ double G[KC][TB + 1];   // A_{k1,k0}: [t][row] of the chunk
  __shared__ double Bk[KC][64 + 1];  // panel k0, rows t of the chunk, columns c0 ..
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  double acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[i][q] = 0.0;
  for (int tc = 0; tc < TB; tc += KC) {
    for (int e = tid; e < KC * TB; e += 256) {
      const int r = e / KC, t = e % KC;
      G[t][r] = A[(int64_t)(k1 * TB + r) * ld + k0 * TB + tc + t];
    }
    for (int e = tid; e < KC * 64; e += 256) {
      const int t = e / 64, cc = e % 64;
      Bk[t][cc] = A[(int64_t)(k0 * TB + tc + t) * ld + c0 + cc];
    }
    __syncthreads();
#pragma unroll 4
    for (int t = 0; t < KC; ++t)
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[i][q] = fma(G[t][ty * 8 + i], Bk[t][tx * 4 + q], acc[i][q]);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int col = c0 + tx * 4 + q;
      if (col >= k1 * TB) continue;
      const int64_t idx = (int64_t)(k1 * TB + ty * 8 + i) * ld + col;
      // j < 2u: the original block plus the product; j = 2u: the product alone
      out[idx] = (col < k0 * TB ? A[idx] : 0.0) + acc[i][q];
    }
}

template <bool TF32>
__global__ void split_aop_kernel(const double* __restrict__ A, int64_t count, void* __restrict__ hi,
                                 void* __restrict__ lo) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const double a = A[e];
    if constexpr (TF32) {
      uint32_t hb;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hb) : "f"((float)a));
      const float h = __uint_as_float(hb);
      static_cast<float*>(hi)[e] = h;
      static_cast<float*>(lo)[e] = (float)(a - (double)h);
    } else {
      const __nv_bfloat16 h = __double2bfloat16(a);
      static_cast<__nv_bfloat16*>(hi)[e] = h;
      static_cast<__nv_bfloat16*>(lo)[e] = __double2bfloat16(a - (double)__bfloat162float(h));
    }
  }
}

// ------------------------------------------------------------------- host side

struct TcState {
  bool tf32 = false;
  int n = 0, n_pad = 0, bs = 0, P = 0, num_sms = 0;
  void* ahi = nullptr;
  void* alo = nullptr;
  float* xt32 = nullptr;
  void* bhi = nullptr;
  void* blo = nullptr;
  int64_t ldt = 0;
  int8_t* shift = nullptr;        // per-SNP integer shift (bs) of the last block: one of shift_buf
  int8_t* shift_buf[2] = {nullptr, nullptr};  // inverse form: alternate blocks (a block's shifts stay
  int shift_slot = 0;                         // intact while the next block is cast)
  bool center = false;            // X_L[:, 0] is the intercept: shift SNP columns
  int strip_group = 0;            // tile order over groups of column strips (0: all)
  TileMode mode = TILES_SINGLE;    // how tiles map onto CTAs
  int max_clusters = 0;            // pair modes: co-resident 2-CTA clusters of the kernel
  uint32_t* order = nullptr;      // device tile order when strip_group > 0
  int order_C = -1;               // the column-strip count the order was built for
  unsigned int* sched = nullptr;  // [0] counter, flags from +32
  size_t sched_bytes = 0;
  DevStatus* st = nullptr;
  CUtensorMap mAhi, mAlo, mBhi, mBlo, mBhiH, mBloH;
  CUtensorMap mStX, mStHi, mStLo;  // pair product's epilogue stores
  CUtensorMap mRed;                // the reduction's view of the FP32 X~ (box RED_BOX_ROWS x RED_BOX_COLS)
  void* xc = nullptr;  // inverse form: the cast block x - c_i (n_pad x bs, BF16, FP32 or FP16)
  bool f16 = false;           // inverse form with FP16 pieces of L^-1 (row-scaled) and an FP16 cast block
  float* rscale = nullptr;    // f16: per-row scale of L^-1 (n_pad)
  // inverse form: the per-SNP sums fused into the launch (set_reductions)
  const float* w32 = nullptr;  // W in FP32, row-major, row stride ws
  int ws = 0, nw = 0;
  float* red = nullptr;        // partials: P (ws 4) or 4P (ws 8) groups of nw + 1 planes of bs floats
  bool red_last = false;       // the last block's sums are in red
  EncodeTiledFn encode = nullptr;
};

// Row entries of the tile order: row panels, or row-panel pairs in pair mode.
static int unit_rows(const TcState* t) { return t->mode == TILES_SINGLE ? t->P : (t->P + 1) / 2; }

cudaError_t get_encode(EncodeTiledFn* fn) {
  void* f = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess) return e;
  if (q != cudaDriverEntryPointSuccess || !f) return cudaErrorNotSupported;
  *fn = reinterpret_cast<EncodeTiledFn>(f);
  return cudaSuccess;
}

// 2D tiled map: dims {inner, outer}, outer stride in bytes, box {bi, bo};
// swz: the 64-byte swizzle of the operand stages (box inner extent 64 bytes).
cudaError_t make_map(EncodeTiledFn enc, CUtensorMap* m, CUtensorMapDataType dt, const void* base,
                            uint64_t inner, uint64_t outer, uint64_t stride_bytes, uint32_t bi, uint32_t bo,
                            bool swz) {
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {stride_bytes};
  cuuint32_t box[2] = {bi, bo};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(m, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   swz ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

static cudaError_t build_inverse(TcState* t, const double* Aop, cudaStream_t s, int64_t* launches);

cudaError_t create(TcState** out, Split split, const double* Aop, int n, int n_pad, int bs, int num_sms,
                   bool center, DevStatus* st, cudaStream_t s, int64_t* launches, int strip_group, TileMode mode) {
  *out = nullptr;
  if (mode != TILES_AUTO && mode != TILES_SINGLE && mode != TILES_PAIR_MMA && mode != TILES_INVERSE)
    return cudaErrorInvalidValue;
  if (split == SPLIT_F16 && mode != TILES_AUTO && mode != TILES_INVERSE) return cudaErrorInvalidValue;
  TcState* t = new TcState;
  t->tf32 = (split == SPLIT_TF32);
  t->f16 = (split == SPLIT_F16);  // otherwise BF16
  t->n = n;
  t->n_pad = n_pad;
  t->bs = bs;
  t->P = n_pad / TB;
  t->num_sms = num_sms;
  t->st = st;
  t->ldt = n_pad;
  const size_t esz = t->tf32 ? 4 : 2;
  const size_t n2 = (size_t)n_pad * n_pad;
  const int Cmax = (bs + TN - 1) / TN;
  cudaError_t e;
#define TRY(x)              \
  do {                      \
    e = (x);                \
    if (e != cudaSuccess) { \
      destroy(t);           \
      return e;             \
    }                       \
  } while (0)
  TRY(get_encode(&t->encode));
  TRY(cudaMalloc(&t->ahi, esz * n2));
  TRY(cudaMalloc(&t->alo, esz * n2));
  TRY(cudaMalloc(&t->xt32, sizeof(float) * (size_t)n_pad * bs));
  if (!t->tf32) TRY(cudaMalloc(&t->bhi, 2 * (size_t)n_pad * bs));
  TRY(cudaMalloc(&t->blo, esz * (size_t)n_pad * bs));
  TRY(cudaMalloc(&t->shift_buf[0], 2 * (size_t)bs));
  t->shift_buf[1] = t->shift_buf[0] + bs;
  t->shift = t->shift_buf[0];
  t->center = center;
  t->strip_group = strip_group;
  // measured at n = 1e4 with 4096-column blocks: the inverse form is the
  // fastest for both splits (BF16: 0.51 ms a block against 0.93 ms for the
  // pair product of the substitution)
  if (mode == TILES_AUTO) mode = TILES_INVERSE;
  t->mode = mode;
  const bool inv = mode == TILES_INVERSE;
  if (inv) TRY(cudaMalloc(&t->xc, esz * (size_t)n_pad * bs));
  if (t->f16) TRY(cudaMalloc(&t->rscale, sizeof(float) * (size_t)n_pad));
  if (strip_group > 0 || inv) {
    TRY(cudaMalloc(&t->order, sizeof(uint32_t) * (size_t)t->P * Cmax));
  }
  t->sched_bytes = 128 + sizeof(int) * (size_t)t->P * Cmax;
  TRY(cudaMalloc(&t->sched, t->sched_bytes));
  TRY(cudaMemsetAsync(t->sched, 0, t->sched_bytes, s));
  if (inv) {
    TRY(build_inverse(t, Aop, s, launches));
  } else {
    // the pair product multiplies the pair form of the operator (pair_rows_kernel)
    const double* src = Aop;
    double* pair_form = nullptr;
    if (mode == TILES_PAIR_MMA && t->P > 1) {
      TRY(cudaMallocAsync(&pair_form, sizeof(double) * n2, s));
      TRY(cudaMemcpyAsync(pair_form, Aop, sizeof(double) * n2, cudaMemcpyDeviceToDevice, s));
      pair_rows_kernel<<<dim3(n_pad / 64, t->P / 2), 256, 0, s>>>(Aop, pair_form, n_pad, t->P);
      ++*launches;
      TRY(cudaGetLastError());
      src = pair_form;
    }
    if (t->tf32)
      split_aop_kernel<true><<<1184, 256, 0, s>>>(src, (int64_t)n2, t->ahi, t->alo);
    else
      split_aop_kernel<false><<<1184, 256, 0, s>>>(src, (int64_t)n2, t->ahi, t->alo);
    ++*launches;
    if (pair_form) TRY(cudaFreeAsync(pair_form, s));
    TRY(cudaGetLastError());
  }
  const CUtensorMapDataType dt = t->tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const CUtensorMapDataType dta = t->f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : dt;  // the operator pieces
  const uint32_t kch = t->tf32 ? Cfg<true>::KCH : Cfg<false>::KCH;
  TRY(make_map(t->encode, &t->mAhi, dta, t->ahi, n_pad, n_pad, esz * n_pad, kch, TB, true));
  TRY(make_map(t->encode, &t->mAlo, dta, t->alo, n_pad, n_pad, esz * n_pad, kch, TB, true));
  const void* bhi_base = t->tf32 ? static_cast<const void*>(t->xt32) : t->bhi;
  TRY(make_map(t->encode, &t->mBhi, dt, bhi_base, n_pad, bs, esz * n_pad, kch, TN, true));
  TRY(make_map(t->encode, &t->mBlo, dt, t->blo, n_pad, bs, esz * n_pad, kch, TN, true));
  TRY(make_map(t->encode, &t->mBhiH, dt, bhi_base, n_pad, bs, esz * n_pad, kch, TN / 2, true));
  TRY(make_map(t->encode, &t->mBloH, dt, t->blo, n_pad, bs, esz * n_pad, kch, TN / 2, true));
  // epilogue store chunks: the pair product's (value + pieces in one 2 KB
  // buffer), or the inverse form's (FP32 value alone, 16 columns)
  const uint32_t stc = inv ? inv2::ST_COLS : (t->tf32 ? pair2::st_cols<true>() : pair2::st_cols<false>());
  TRY(make_map(t->encode, &t->mRed, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, t->xt32, n_pad, bs, 4 * (size_t)n_pad,
               RED_BOX_ROWS, RED_BOX_COLS, false));
  TRY(make_map(t->encode, &t->mStX, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, t->xt32, n_pad, bs, 4 * (size_t)n_pad, 32, stc,
               false));
  memset(&t->mStHi, 0, sizeof t->mStHi);
  if (!t->tf32) TRY(make_map(t->encode, &t->mStHi, dt, t->bhi, n_pad, bs, esz * n_pad, 32, stc, false));
  TRY(make_map(t->encode, &t->mStLo, dt, t->blo, n_pad, bs, esz * n_pad, 32, stc, false));
  TRY(set_kernel_attrs(t->tf32, mode != TILES_SINGLE));
  if (mode != TILES_SINGLE) {
    TRY(query_clusters(t->tf32, mode, num_sms, &t->max_clusters, t->f16));
    if (t->max_clusters < 1) TRY(cudaErrorLaunchOutOfResources);
  }
#undef TRY
  *out = t;
  return cudaSuccess;
}

// Tile order of one study: row panel by row panel over groups of G column
// strips (G <= 0 or G >= C: all strips), study index `si` in the top bits.
static void append_study_order(std::vector<uint32_t>& order, int si, int P, int C, int G) {
  if (G <= 0 || G > C) G = C;
  for (int c0 = 0; c0 < C; c0 += G)
    for (int k = 0; k < P; ++k)
      for (int c = c0; c < c0 + G && c < C; ++c)
        order.push_back(((uint32_t)si << 28) | ((uint32_t)k << 14) | (uint32_t)c);
}

// Inverse form: work units longest first (pair row r has 2r + 2 K-blocks, the
// last row of an odd P 2r + 1), the studies' units merged by length; equal
// lengths keep study, then strip order.
struct UnitKey {
  int len;
  uint32_t code;
};
// The inverse form's units with their K-block counts (the device's
// pair2::make_unit_inv: with an odd P the lone panel is panel 0).
static void append_units(std::vector<UnitKey>& v, int si, int P, int C) {
  const int o = P & 1;
  for (int r = 0; r < (P + 1) / 2; ++r) {
    const int k0 = (o && r == 0) ? 0 : 2 * r - o;
    const int len = (o && r == 0) ? 1 : k0 + (k0 + 1 < P ? 2 : 1);
    for (int c = 0; c < C; ++c) v.push_back({len, ((uint32_t)si << 28) | ((uint32_t)r << 14) | (uint32_t)c});
  }
}
static void longest_first(std::vector<UnitKey>& v, std::vector<uint32_t>& order) {
  std::stable_sort(v.begin(), v.end(), [](const UnitKey& a, const UnitKey& b) { return a.len > b.len; });
  for (const UnitKey& u : v) order.push_back(u.code);
}

static int cast_out(const TcState* t) { return t->tf32 ? OUT_F32 : (t->f16 ? OUT_F16 : OUT_BF16); }
bool packed_ok(const TcState* t);

// Inverse form: the cast block's map (half-width boxes) and the cast
// pre-pass (with the integer shifts when centering).
static cudaError_t prepare_cast(TcState* t, const int8_t* X, int64_t ldx, int ncols, cudaStream_t s,
                                int64_t* launches, CUtensorMap* mXcH, bool packed = false) {
  const size_t esz = t->tf32 ? 4 : 2;
  const CUtensorMapDataType dt = t->tf32  ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : t->f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                          : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const uint32_t kch = t->tf32 ? Cfg<true>::KCH : Cfg<false>::KCH;
  cudaError_t e = make_map(t->encode, mXcH, dt, t->xc, (uint64_t)t->n_pad, (uint64_t)ncols, esz * t->n_pad, kch,
                           TN / 2, true);
  if (e != cudaSuccess) return e;
  if (t->center) {  // this block's shift slot
    t->shift_slot ^= 1;
    t->shift = t->shift_buf[t->shift_slot];
  }
  int8_t* sh = t->center ? t->shift : nullptr;
  ++*launches;
  if ((e = launch_cast(cast_out(t), X, ldx, t->n, t->n_pad, ncols, sh, t->xc, t->sched, s, packed)) != cudaSuccess)
    return e;
  return cudaGetLastError();
}

// The study part of one launch: int8 map, cleared flags, integer shifts.
static cudaError_t prepare_study(TcState* t, const int8_t* X, int64_t ldx, int ncols, cudaStream_t s,
                                 int64_t* launches, TcStudy* S, CUtensorMap* mX8, CUtensorMap* mX8H,
                                 CUtensorMap* mXcH, bool packed = false) {
  if (ncols > t->bs || (reinterpret_cast<uintptr_t>(X) & 15) || (ldx & 15) || ldx < (packed ? (t->n + 3) / 4 : t->n))
    return cudaErrorInvalidValue;
  if (packed && !packed_ok(t)) return cudaErrorInvalidValue;
  cudaError_t e;
  if (t->mode != TILES_INVERSE) {
    e = make_map(t->encode, mX8, CU_TENSOR_MAP_DATA_TYPE_UINT8, X, (uint64_t)t->n, (uint64_t)ncols, (uint64_t)ldx, TB,
                 TN, false);
    if (e != cudaSuccess) return e;
    e = make_map(t->encode, mX8H, CU_TENSOR_MAP_DATA_TYPE_UINT8, X, (uint64_t)t->n, (uint64_t)ncols, (uint64_t)ldx,
                 TB, TN / 2, false);
    if (e != cudaSuccess) return e;
  }
  const int C = (ncols + TN - 1) / TN;
  // the substitution's counter and tile flags; the inverse form uses the
  // counter alone, which its cast zeroes (no stream operation between the
  // previous block's kernels and this cast)
  if (t->mode != TILES_INVERSE && (e = cudaMemsetAsync(t->sched, 0, 128 + sizeof(int) * (size_t)t->P * C, s)) !=
                                      cudaSuccess)
    return e;
  if (t->mode == TILES_INVERSE) {
    if ((e = prepare_cast(t, X, ldx, ncols, s, launches, mXcH, packed)) != cudaSuccess) return e;
  } else if (t->center) {
    column_shift_kernel<<<(ncols + 7) / 8, 256, 0, s>>>(X, ldx, t->n, ncols, t->shift);
    ++*launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  S->P = t->P;
  S->C = C;
  S->ncols = ncols;
  S->n = t->n;
  S->shift = t->center ? t->shift : nullptr;
  S->flags = reinterpret_cast<int*>(t->sched + 32);
  S->xt32 = t->xt32;
  S->bhi = t->bhi;
  S->blo = t->blo;
  S->ldt = t->ldt;
  S->rscale = t->f16 ? t->rscale : nullptr;
  S->w32 = t->w32;
  S->red = t->red;
  S->ws = t->ws;
  S->nw = t->nw;
  S->ldr = t->bs;
  return cudaSuccess;
}

// b.ntiles work units: tiles, or (cluster modes) row-panel pairs of a strip.
static cudaError_t launch_kernel(bool tf32, TileMode mode, const TcBatch& b, int num_sms, int max_clusters,
                                 cudaStream_t s, int64_t* launches, bool f16 = false, int stages = 8) {
  ++*launches;
  return launch_solve(tf32, mode, b, num_sms, max_clusters, s, f16, stages);
}

bool packed_ok(const TcState* t) { return t->mode == TILES_INVERSE && t->n <= 512 * 32; }

cudaError_t run_block(TcState* t, const int8_t* X, int64_t ldx, int ncols, cudaStream_t s, int64_t* launches,
                      cudaEvent_t ev0, cudaEvent_t ev1, bool packed) {
  if (ncols <= 0) return cudaSuccess;
  TcBatch b;
  memset(&b, 0, sizeof b);
  cudaError_t e = prepare_study(t, X, ldx, ncols, s, launches, &b.s0, &b.maps[0].X8, &b.maps[0].X8H, &b.maps[0].XcH,
                                packed);
  if (e != cudaSuccess) return e;
  b.maps[0].Ahi = t->mAhi;
  b.maps[0].Alo = t->mAlo;
  b.maps[0].Bhi = t->mBhi;
  b.maps[0].Blo = t->mBlo;
  b.maps[0].BhiH = t->mBhiH;
  b.maps[0].BloH = t->mBloH;
  b.maps[0].StX = t->mStX;
  b.maps[0].StHi = t->mStHi;
  b.maps[0].StLo = t->mStLo;
  b.nstudies = 1;
  b.ntiles = unit_rows(t) * b.s0.C;
  b.counter = t->sched;
  b.st = t->st;
  t->red_last = b.s0.red != nullptr;
  const bool inv = t->mode == TILES_INVERSE;
  if (inv || (t->strip_group > 0 && t->strip_group < b.s0.C)) {
    if (t->order_C != b.s0.C) {  // (re)build the order for this strip count
      std::vector<uint32_t> order;
      if (inv) {
        std::vector<UnitKey> units;
        append_units(units, 0, t->P, b.s0.C);
        longest_first(units, order);
      } else {
        append_study_order(order, 0, unit_rows(t), b.s0.C, t->strip_group);
      }
      if ((e = cudaMemcpyAsync(t->order, order.data(), sizeof(uint32_t) * order.size(), cudaMemcpyHostToDevice, s)) !=
              cudaSuccess ||
          (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return e;
      t->order_C = b.s0.C;
    }
    b.order = t->order;  // the study descriptor stays b.s0 (studies null)
  }
  if (ev0 && (e = cudaEventRecord(ev0, s)) != cudaSuccess) return e;
  if ((e = launch_kernel(t->tf32, t->mode, b, t->num_sms, t->max_clusters, s, launches, t->f16)) != cudaSuccess)
    return e;
  return ev1 ? cudaEventRecord(ev1, s) : cudaSuccess;
}

// Inverse form set-up: L^-1 = the substitution applied to the identity, on
// the tensor cores in TF32x3 (the pair product over Aop, 4096 identity
// columns per launch, no centering), then transposed and split into the
// row-major hi/lo pieces of t.  Synchronizes the stream.
// L^-1 in FP64: the FP64 blocked solve of int8 identity columns, 4096 at a
// time (tiles above each strip's first column are zero and skipped: n^3/3
// flop in all), then its hi/lo pieces.
static cudaError_t build_inverse(TcState* t, const double* Aop, cudaStream_t s, int64_t* launches) {
  const int np = t->n_pad;
  const int bsi = np < 4096 ? np : 4096;
  const int C64 = (bsi + F64_TN - 1) / F64_TN;
  const size_t sched_bytes = sizeof(Sched) + sizeof(int) * (size_t)t->P * C64;
  int8_t* eye = nullptr;
  double* x64 = nullptr;     // the solved columns, n_pad x bsi
  Sched* sch = nullptr;      // the FP64 solve's counter and tile flags
  double* rows64 = nullptr;  // FP16 pieces: the whole L^-1, row-major, before the row scales are known
  cudaError_t e = cudaMalloc(&eye, (size_t)np * bsi);
  if (e == cudaSuccess) e = cudaMalloc(&x64, sizeof(double) * (size_t)np * bsi);
  if (e == cudaSuccess) e = cudaMalloc(&sch, sched_bytes);
  if (e == cudaSuccess && t->f16) e = cudaMalloc(&rows64, sizeof(double) * (size_t)np * np);
  for (int c0 = 0; e == cudaSuccess && c0 < np; c0 += bsi) {
    const int nc = np - c0 < bsi ? np - c0 : bsi;
    identity_i8_kernel<<<1184, 256, 0, s>>>(eye, np, c0, nc);
    ++*launches;
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(sch, 0, sched_bytes, s)) != cudaSuccess) break;
    TrsmF64Args a{};
    a.Aop = Aop;
    a.lda = np;
    a.X = eye;
    a.ldx = np;
    a.n = t->n;
    a.Xt = x64;
    a.ldt = np;
    a.P = t->P;
    a.ncols = nc;
    a.C = (nc + F64_TN - 1) / F64_TN;
    a.sched = sch;
    a.st = t->st;
    a.tri_col0 = c0;
    if ((e = launch_trsm_f64(a, true, s, t->num_sms)) != cudaSuccess) break;
    ++*launches;
    const dim3 grid((nc + 31) / 32, np / 32);
    if (t->f16)
      linv_rows_kernel<<<grid, dim3(32, 8), 0, s>>>(x64, np, t->n, np, c0, nc, rows64);
    else if (t->tf32)
      linv_split_kernel<true><<<grid, dim3(32, 8), 0, s>>>(x64, np, t->n, np, c0, nc, t->ahi, t->alo);
    else
      linv_split_kernel<false><<<grid, dim3(32, 8), 0, s>>>(x64, np, t->n, np, c0, nc, t->ahi, t->alo);
    ++*launches;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && t->f16) {
    linv_split_f16_kernel<<<np, 256, 0, s>>>(rows64, np, static_cast<__half*>(t->ahi), static_cast<__half*>(t->alo),
                                              t->rscale);
    ++*launches;
    e = cudaGetLastError();
  }
  const cudaError_t es = cudaStreamSynchronize(s);  // before the buffers go
  if (e == cudaSuccess) e = es;
  if (e == cudaSuccess && t->st) {
    DevStatus h;
    if ((e = cudaMemcpy(&h, t->st, sizeof h, cudaMemcpyDeviceToHost)) == cudaSuccess && h.err != DEV_OK)
      e = cudaErrorLaunchTimeout;  // a bounded wait of the solve expired
  }
  cudaFree(eye);
  cudaFree(x64);
  cudaFree(sch);
  cudaFree(rows64);
  return e;
}

cudaError_t set_reductions(TcState* t, const float* w32, int ws, int nw) {
  if (t->red || t->mode != TILES_INVERSE || nw < 1 || nw > 8 || (ws != 4 && ws != 8) || ws < nw) return cudaSuccess;
  cudaError_t e = cudaMalloc(&t->red, sizeof(float) * (size_t)t->P * 4 * (nw + 1) * t->bs);
  if (e != cudaSuccess) return e;
  t->w32 = w32;
  t->ws = ws;
  t->nw = nw;
  return cudaSuccess;
}
cudaError_t drop_lo_piece(TcState* t, cudaStream_t s) {
  if (t->mode != TILES_INVERSE) return cudaErrorInvalidValue;
  const size_t esz = t->tf32 ? 4 : 2;
  return cudaMemsetAsync(t->alo, 0, esz * (size_t)t->n_pad * t->n_pad, s);
}
const float* partials(const TcState* t) { return t->red_last ? t->red : nullptr; }
int partial_groups(const TcState* t) { return t->ws == 4 ? t->P : 4 * t->P; }  // row panels or their quarters
int64_t partial_ld(const TcState* t) { return t->bs; }

// ------------------------------------------------------------- batched launch
struct TcBatchState {
  int nstudies = 0;
  int ntiles = 0;
  TcStudy S[MAX_STUDIES];
  CUtensorMap mX8[MAX_STUDIES], mX8H[MAX_STUDIES], mXcH[MAX_STUDIES] = {};
  const int8_t* X[MAX_STUDIES];
  int64_t ldx[MAX_STUDIES];
  bool tf32 = false, f16 = false;
  TileMode mode = TILES_SINGLE;
  int num_sms = 0, max_clusters = 0;
  int stages = 8;                // operand stages of the inverse-form kernel (8 or 6)
  TcStudy* d_studies = nullptr;  // device copies
  uint32_t* d_order = nullptr;
  unsigned int* d_counter = nullptr;
  size_t order_cap = 0;
  DevStatus* st = nullptr;
};

cudaError_t batch_create(TcBatchState** out, TcState* const* ts, int nstudies) {
  *out = nullptr;
  if (nstudies < 1 || nstudies > MAX_STUDIES) return cudaErrorInvalidValue;
  for (int i = 1; i < nstudies; ++i)
    if (ts[i]->tf32 != ts[0]->tf32 || ts[i]->f16 != ts[0]->f16 || ts[i]->mode != ts[0]->mode)
      return cudaErrorInvalidValue;
  TcBatchState* B = new TcBatchState;
  B->nstudies = nstudies;
  B->tf32 = ts[0]->tf32;
  B->f16 = ts[0]->f16;
  B->mode = ts[0]->mode;
  B->num_sms = ts[0]->num_sms;
  B->max_clusters = ts[0]->max_clusters;
  B->st = ts[0]->st;
  size_t cap = 0;
  for (int i = 0; i < nstudies; ++i) cap += (size_t)unit_rows(ts[i]) * ((ts[i]->bs + TN - 1) / TN);
  B->order_cap = cap;
  cudaError_t e;
  if ((e = cudaMalloc(&B->d_studies, sizeof(TcStudy) * MAX_STUDIES)) != cudaSuccess ||
      (e = cudaMalloc(&B->d_order, sizeof(uint32_t) * cap)) != cudaSuccess ||
      (e = cudaMalloc(&B->d_counter, 128)) != cudaSuccess) {
    batch_destroy(B);
    return e;
  }
  *out = B;
  return cudaSuccess;
}

// Fixes the launch geometry: the study descriptors and the tile order
// (order_mode 0: row panel by row panel across the studies; 1: study after
// study).  Synchronizes the stream (host copies).  The X pointers are the
// device blocks later launches will read.
cudaError_t batch_plan(TcBatchState* B, TcState* const* ts, const int8_t* const* X, const int64_t* ldx,
                       const int* ncols, int order_mode, cudaStream_t s, int strip_group) {
  TcStudy S[MAX_STUDIES];
  memset(S, 0, sizeof S);
  int pmax = 0, total = 0;
  for (int i = 0; i < B->nstudies; ++i) {
    TcState* t = ts[i];
    if (ncols[i] < 0 || ncols[i] > t->bs) return cudaErrorInvalidValue;
    if (ncols[i] == 0) continue;
    if ((reinterpret_cast<uintptr_t>(X[i]) & 15) || (ldx[i] & 15) || ldx[i] < t->n) return cudaErrorInvalidValue;
    cudaError_t e = make_map(t->encode, &B->mX8[i], CU_TENSOR_MAP_DATA_TYPE_UINT8, X[i], (uint64_t)t->n,
                             (uint64_t)ncols[i], (uint64_t)ldx[i], TB, TN, false);
    if (e != cudaSuccess) return e;
    e = make_map(t->encode, &B->mX8H[i], CU_TENSOR_MAP_DATA_TYPE_UINT8, X[i], (uint64_t)t->n, (uint64_t)ncols[i],
                 (uint64_t)ldx[i], TB, TN / 2, false);
    if (e != cudaSuccess) return e;
    if (t->mode == TILES_INVERSE) {
      const size_t esz = t->tf32 ? 4 : 2;
      e = make_map(t->encode, &B->mXcH[i],
                   t->tf32  ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                   : t->f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                            : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                   t->xc,
                   (uint64_t)t->n_pad, (uint64_t)ncols[i], esz * t->n_pad, t->tf32 ? Cfg<true>::KCH : Cfg<false>::KCH,
                   TN / 2, true);
      if (e != cudaSuccess) return e;
    }
    S[i].P = t->P;
    S[i].C = (ncols[i] + TN - 1) / TN;
    S[i].ncols = ncols[i];
    S[i].n = t->n;
    S[i].shift = t->center ? t->shift : nullptr;
    S[i].flags = reinterpret_cast<int*>(t->sched + 32);
    S[i].xt32 = t->xt32;
    S[i].bhi = t->bhi;
    S[i].blo = t->blo;
    S[i].ldt = t->ldt;
    S[i].rscale = t->f16 ? t->rscale : nullptr;
    S[i].w32 = t->w32;
    S[i].red = t->red;
    S[i].ws = t->ws;
    S[i].nw = t->nw;
    S[i].ldr = t->bs;
    t->red_last = ncols[i] > 0 && t->red != nullptr;
    pmax = unit_rows(t) > pmax ? unit_rows(t) : pmax;
    total += unit_rows(t) * S[i].C;
  }
  std::vector<uint32_t> order;
  order.reserve(total);
  if (B->mode == TILES_INVERSE) {  // no dependencies: longest units first over all studies
    std::vector<UnitKey> units;
    for (int i = 0; i < B->nstudies; ++i)
      if (ncols[i] > 0) append_units(units, i, ts[i]->P, S[i].C);
    longest_first(units, order);
  } else if (order_mode == 0) {
    for (int k = 0; k < pmax; ++k)
      for (int i = 0; i < B->nstudies; ++i)
        if (ncols[i] > 0 && k < unit_rows(ts[i]))
          for (int c = 0; c < S[i].C; ++c) order.push_back(((uint32_t)i << 28) | ((uint32_t)k << 14) | (uint32_t)c);
  } else {
    for (int i = 0; i < B->nstudies; ++i)
      if (ncols[i] > 0) append_study_order(order, i, unit_rows(ts[i]), S[i].C, strip_group);
  }
  cudaError_t e;
  if (total > 0 &&
      (e = cudaMemcpyAsync(B->d_order, order.data(), sizeof(uint32_t) * order.size(), cudaMemcpyHostToDevice, s)) !=
          cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(B->d_studies, S, sizeof(TcStudy) * MAX_STUDIES, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  memcpy(B->S, S, sizeof S);
  memcpy(B->X, X, sizeof(const int8_t*) * B->nstudies);
  memcpy(B->ldx, ldx, sizeof(int64_t) * B->nstudies);
  B->ntiles = total;
  return cudaSuccess;
}

// One planned launch: clear flags and counter, shift pre-passes, the batched
// kernel.  Only stream-ordered work: can be captured into a CUDA graph.
cudaError_t batch_launch(TcBatchState* B, TcState* const* ts, cudaStream_t s, int64_t* launches) {
  if (B->ntiles == 0) return cudaSuccess;
  TcBatch b;
  memset(&b, 0, sizeof b);
  cudaError_t e;
  // inverse form with every study at n <= 16384: the casts in one launch, which
  // also zeroes the counter (the inverse form's tiles use no flags)
  int nmax = 0;
  for (int i = 0; i < B->nstudies; ++i)
    if (B->S[i].ncols > 0) nmax = std::max(nmax, ts[i]->n);
  const bool one_cast = B->mode == TILES_INVERSE && nmax <= 512 * 32;
  CastJobs J;
  memset(&J, 0, sizeof J);
  J.counter = B->d_counter;
  for (int i = 0; i < B->nstudies; ++i) {
    if (B->S[i].ncols == 0) continue;
    TcState* t = ts[i];
    if (one_cast) {  // cast below, with every study's columns
      J.j[J.njobs++] = CastJob{B->X[i], B->ldx[i], t->n, t->n_pad, J.total, B->S[i].ncols,
                               t->center ? t->shift : nullptr, t->xc};
      J.total += B->S[i].ncols;
    } else if ((e = cudaMemsetAsync(t->sched, 0, 128 + sizeof(int) * (size_t)t->P * B->S[i].C, s)) != cudaSuccess) {
      return e;
    } else if (t->mode == TILES_INVERSE) {
      int8_t* sh = t->center ? t->shift : nullptr;
      ++*launches;
      if ((e = launch_cast(cast_out(t), B->X[i], B->ldx[i], t->n, t->n_pad, B->S[i].ncols, sh, t->xc, nullptr, s)) !=
          cudaSuccess)
        return e;
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    } else if (t->center) {
      column_shift_kernel<<<(B->S[i].ncols + 7) / 8, 256, 0, s>>>(B->X[i], B->ldx[i], t->n, B->S[i].ncols, t->shift);
      ++*launches;
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    b.maps[i].Ahi = t->mAhi;
    b.maps[i].Alo = t->mAlo;
    b.maps[i].Bhi = t->mBhi;
    b.maps[i].Blo = t->mBlo;
    b.maps[i].X8 = B->mX8[i];
    b.maps[i].BhiH = t->mBhiH;
    b.maps[i].BloH = t->mBloH;
    b.maps[i].X8H = B->mX8H[i];
    b.maps[i].XcH = B->mXcH[i];
    b.maps[i].StX = t->mStX;
    b.maps[i].StHi = t->mStHi;
    b.maps[i].StLo = t->mStLo;
  }
  if (one_cast) {
    const int out = cast_out(ts[0]);  // one split for the whole batch
    e = out == OUT_F32   ? launch_cast_batch_t<OUT_F32>(J, nmax, s)
        : out == OUT_F16 ? launch_cast_batch_t<OUT_F16>(J, nmax, s)
                         : launch_cast_batch_t<OUT_BF16>(J, nmax, s);
    if (e != cudaSuccess) return e;
    ++*launches;
  } else if ((e = cudaMemsetAsync(B->d_counter, 0, 128, s)) != cudaSuccess) {
    return e;
  }
  b.studies = B->d_studies;
  b.order = B->d_order;
  b.nstudies = B->nstudies;
  b.ntiles = B->ntiles;
  b.counter = B->d_counter;
  b.st = B->st;
  return launch_kernel(B->tf32, B->mode, b, B->num_sms, B->max_clusters, s, launches, B->f16, B->stages);
}

cudaError_t batch_set_stages(TcBatchState* B, int stages) {
  if (stages != 6 && stages != 8) return cudaErrorInvalidValue;
  B->stages = stages;
  return cudaSuccess;
}

void batch_destroy(TcBatchState* B) {
  if (!B) return;
  cudaFree(B->d_studies);
  cudaFree(B->d_order);
  cudaFree(B->d_counter);
  delete B;
}

const float* xt_f32(const TcState* t) { return t->xt32; }
const CUtensorMap* xt_reduce_map(const TcState* t) { return &t->mRed; }
const int8_t* shift_of(const TcState* t) { return t->center ? t->shift : nullptr; }
int64_t xt_ld(const TcState* t) { return t->ldt; }
TileMode tile_mode(const TcState* t) { return t->mode; }

void launch_shape(const TcState* t, int* ctas, int* cluster_size) {
  const int units = unit_rows(t) * ((t->bs + TN - 1) / TN);
  if (t->mode == TILES_SINGLE) {
    *ctas = units < t->num_sms ? units : t->num_sms;
    *cluster_size = 1;
  } else {
    *ctas = 2 * (units < t->max_clusters ? units : t->max_clusters);
    *cluster_size = 2;
  }
}

void destroy(TcState* t) {
  if (!t) return;
  cudaFree(t->red);
  cudaFree(t->ahi);
  cudaFree(t->alo);
  cudaFree(t->xt32);
  cudaFree(t->bhi);
  cudaFree(t->blo);
  cudaFree(t->xc);
  cudaFree(t->rscale);
  cudaFree(t->sched);
  cudaFree(t->shift_buf[0]);
  cudaFree(t->order);
  delete t;
}
}  // namespace tc
}  // namespace gwas
