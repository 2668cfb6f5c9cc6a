// 2-bit packed SNP columns: hard-called genotypes (values 0..3) four to a
// byte, the way genotype files commonly store them.  The host link, not the
// solve, bounds the whole-study stream of int8 columns (n bytes per SNP at
// ~56 GB/s against ~7.6 M SNPs/s of solves at n = 10^4); columns that are
// already packed cross it in a quarter of the bytes and are unpacked in HBM
// (gwas_solve_stream_packed).  Packing on the host in the stream itself does
// not pay: 16 host cores pack ~20 GB/s of int8, below the link's 56 GB/s.
//
// Encoding (gwas_pack_dosages2): column c occupies ceil(n/4) bytes at P + c ldp;
// byte k holds rows 4k .. 4k+3, row 4k + i in bits 2i .. 2i+1; rows past n are 0.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>

#include "gwas_internal.cuh"

namespace gwas {

// ---------------------------------------------------------------- packing
// Eight rows a step: bytes b0..b7 of a little-endian word (each 0..3) fold to
// the two packed bytes (b0 | b1 << 2 | b2 << 4 | b3 << 6) and the same of b4..b7.
static inline uint16_t pack8(uint64_t w) {
  uint64_t v = (w | (w >> 6)) & 0x000F000F000F000Full;  // nibbles b0|b1<<2 at bits 0, 16, 32, 48
  v = (v | (v >> 12)) & 0x000000FF000000FFull;          // bytes at bits 0 and 32
  return (uint16_t)(v | (v >> 24));
}

bool pack2_columns(const int8_t* X, int64_t ldx, int n, int c0, int c1, uint8_t* P, int64_t ldp) {
  const int nb = (n + 3) / 4;
  for (int c = c0; c < c1; ++c) {
    const uint8_t* x = reinterpret_cast<const uint8_t*>(X + (int64_t)c * ldx);
    uint8_t* o = P + (int64_t)c * ldp;
    uint64_t bad = 0;
    int r = 0;
    for (; r + 8 <= n; r += 8) {
      uint64_t w;
      std::memcpy(&w, x + r, 8);
      bad |= w;
      const uint16_t h = pack8(w);
      std::memcpy(o + r / 4, &h, 2);
    }
    if (r < n) {  // the ragged end: rows past n count as 0
      uint8_t t[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      std::memcpy(t, x + r, (size_t)(n - r));
      uint64_t w;
      std::memcpy(&w, t, 8);
      bad |= w;
      const uint16_t h = pack8(w);
      const int left = nb - r / 4;  // 1 or 2 bytes of this column remain
      std::memcpy(o + r / 4, &h, (size_t)left);
    }
    if (bad & 0xFCFCFCFCFCFCFCFCull) return false;  // a value outside 0..3
  }
  return true;
}

// --------------------------------------------------------------- unpacking
// One thread per 4 packed bytes (16 rows of a column): a 16-byte store of
// the int8 values.  X rows 16 t .. 16 t + 15 < ceil(n / 16) 16 <= n_pad; rows
// past n come out 0, as the slot holds them.
__global__ void unpack2_kernel(const uint8_t* __restrict__ P, int64_t ldp, int n, int ncols, int8_t* __restrict__ X,
                               int64_t ldx) {
  const int col = blockIdx.y;
  const int g = blockIdx.x * blockDim.x + threadIdx.x;  // group of 16 rows
  if (col >= ncols || 16 * g >= n) return;
  const uint8_t* p = P + (int64_t)col * ldp + 4 * g;
  const int nb = (n + 3) / 4;  // packed bytes of the column
  uint32_t v = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (4 * g + k < nb) v |= (uint32_t)p[k] << (8 * k);
  uint32_t w[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint32_t b = (v >> (8 * k)) & 0xFFu;  // rows 16g + 4k .. +3
    w[k] = (b & 3u) | ((b & 0xCu) << 6) | ((b & 0x30u) << 12) | ((b & 0xC0u) << 18);
  }
  if (16 * g + 16 > n)  // rows past n as 0, whatever bits the packed padding holds
    for (int i = 0; i < 16; ++i)
      if (16 * g + i >= n) w[i >> 2] &= ~(0xFFu << (8 * (i & 3)));
  *reinterpret_cast<uint4*>(X + (int64_t)col * ldx + 16 * g) = make_uint4(w[0], w[1], w[2], w[3]);
}

cudaError_t launch_unpack2(const uint8_t* P, int64_t ldp, int n, int ncols, int8_t* X, int64_t ldx, cudaStream_t s) {
  if (ncols <= 0) return cudaSuccess;
  if ((ldx & 15) || (reinterpret_cast<uintptr_t>(X) & 15) || ldx < (n + 15) / 16 * 16) return cudaErrorInvalidValue;
  const int groups = (n + 15) / 16;
  unpack2_kernel<<<dim3((groups + 127) / 128, ncols), 128, 0, s>>>(P, ldp, n, ncols, X, ldx);
  return cudaGetLastError();
}

}  // namespace gwas

extern "C" int gwas_pack_dosages2(const int8_t* X, int64_t ldx, int n, int ncols, uint8_t* P, int64_t ldp) {
  if (!X || !P || n < 1 || ncols < 0 || ldx < n || ldp < (n + 3) / 4) return GWAS_ERR_ARG;
  return gwas::pack2_columns(X, ldx, n, 0, ncols, P, ldp) ? GWAS_OK : GWAS_ERR_ARG;
}
