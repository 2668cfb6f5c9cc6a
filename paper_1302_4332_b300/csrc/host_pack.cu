// 2-bit packed SNP columns: hard-called genotypes (values 0..3) four to a
// byte, the way genotype files commonly store them.  The host link, not the
// solve, bounds the whole-study stream of int8 columns (n bytes per SNP at
// ~56 GB/s against ~7.6 M SNPs/s of solves at n = 10^4); packed columns cross
// it in a quarter of the bytes and are unpacked in HBM.  Columns that arrive
// packed go straight over (gwas_solve_stream_packed); int8 columns are packed
// by a pool of host threads inside gwas_solve_stream where the host packs
// faster than the link carries int8: with AVX-512 16 host cores pack ~73 GB/s
// of int8, the scalar form ~20 GB/s.
//
// Encoding (gwas_pack_dosages2): column c occupies ceil(n/4) bytes at P + c ldp;
// byte k holds rows 4k .. 4k+3, row 4k + i in bits 2i .. 2i+1; rows past n are 0.
#include <cuda_runtime.h>
#include <immintrin.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

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

// 64 rows a step with AVX-512 (BW, VL): bytes b0..b3 of each 32-bit lane fold
// to b0 + 4 b1 + 16 b2 + 64 b3 by two multiply-adds (bytes by (1, 4), 16-bit
// pairs by (1, 16)) and one byte a lane is kept.  The ragged end is a masked
// load (rows past n read as 0) and a masked store of its ceil((n - r) / 4)
// bytes.  False when a byte is outside 0..3.  With `nt` (o 16-byte aligned)
// the full 16-byte pieces are written with non-temporal stores, which skip
// reading the destination lines first; the caller fences them.
__attribute__((target("avx512f,avx512bw,avx512vl"))) static bool pack2_column_avx512(const uint8_t* x, int n,
                                                                                       uint8_t* o, bool nt) {
  const __m512i w1 = _mm512_set1_epi16(0x0401);
  const __m512i w2 = _mm512_set1_epi32(0x00100001);
  __m512i bad = _mm512_setzero_si512();
  int r = 0;
  for (; r + 64 <= n; r += 64) {
    const __m512i v = _mm512_loadu_si512(x + r);
    bad = _mm512_or_si512(bad, v);
    const __m512i u = _mm512_madd_epi16(_mm512_maddubs_epi16(v, w1), w2);
    if (nt)
      _mm_stream_si128(reinterpret_cast<__m128i*>(o + r / 4), _mm512_cvtepi32_epi8(u));
    else
      _mm_storeu_si128(reinterpret_cast<__m128i*>(o + r / 4), _mm512_cvtepi32_epi8(u));
  }
  if (r < n) {
    const int left = n - r;  // 1 .. 63
    const __m512i v = _mm512_maskz_loadu_epi8((__mmask64)((1ull << left) - 1), x + r);
    bad = _mm512_or_si512(bad, v);
    const __m512i u = _mm512_madd_epi16(_mm512_maddubs_epi16(v, w1), w2);
    _mm_mask_storeu_epi8(o + r / 4, (__mmask16)((1u << ((left + 3) / 4)) - 1), _mm512_cvtepi32_epi8(u));
  }
  return _mm512_test_epi8_mask(bad, _mm512_set1_epi8((char)0xFC)) == 0;
}

static bool have_avx512bw() {
  static const bool h = __builtin_cpu_supports("avx512f") && __builtin_cpu_supports("avx512bw") &&
                        __builtin_cpu_supports("avx512vl");
  return h;
}

bool pack2_columns(const int8_t* X, int64_t ldx, int n, int c0, int c1, uint8_t* P, int64_t ldp) {
  if (have_avx512bw()) {
    const bool nt = (reinterpret_cast<uintptr_t>(P) & 15) == 0 && (ldp & 15) == 0;
    bool ok = true;
    for (int c = c0; c < c1 && ok; ++c)
      ok = pack2_column_avx512(reinterpret_cast<const uint8_t*>(X + (int64_t)c * ldx), n, P + (int64_t)c * ldp, nt);
    if (nt) _mm_sfence();  // the non-temporal stores ordered before whatever signals completion
    return ok;
  }
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

bool host_pack_fast() { return have_avx512bw(); }

// ---------------------------------------------------------- thread pool
// Persistent workers for pack2_columns over column ranges: run() hands out
// chunks of columns through an atomic cursor; the calling thread works too
// and returns when every chunk is done.
struct PackPool {
  std::vector<std::thread> th;
  std::mutex mu;
  std::condition_variable cv_go, cv_done;
  uint64_t gen = 0;
  bool quit = false;
  // the current job
  const int8_t* X = nullptr;
  int64_t ldx = 0, ldp = 0;
  int n = 0, ncols = 0, chunk = 1;
  uint8_t* P = nullptr;
  std::atomic<int> cursor{0}, pending{0};
  std::atomic<bool> ok{true};

  void work() {
    for (;;) {
      const int c = cursor.fetch_add(chunk);
      if (c >= ncols) break;
      const int c1 = std::min(ncols, c + chunk);
      if (!pack2_columns(X, ldx, n, c, c1, P, ldp)) ok.store(false);
    }
  }
  void loop() {
    uint64_t seen = 0;
    for (;;) {
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_go.wait(lk, [&] { return quit || gen != seen; });
        if (quit) return;
        seen = gen;
      }
      work();
      if (pending.fetch_sub(1) == 1) {
        std::lock_guard<std::mutex> lk(mu);
        cv_done.notify_all();
      }
    }
  }
  bool run(const int8_t* X_, int64_t ldx_, int n_, int ncols_, uint8_t* P_, int64_t ldp_) {
    {
      std::lock_guard<std::mutex> lk(mu);
      X = X_, ldx = ldx_, n = n_, ncols = ncols_, P = P_, ldp = ldp_;
      chunk = std::max(1, ncols_ / (8 * ((int)th.size() + 1)));
      cursor.store(0);
      ok.store(true);
      pending.store((int)th.size());
      ++gen;
    }
    cv_go.notify_all();
    work();
    std::unique_lock<std::mutex> lk(mu);
    cv_done.wait(lk, [&] { return pending.load() == 0; });
    return ok.load();
  }
};

void pack_pool_destroy(PackPool* p);

// Null when the threads cannot be started (nothing is left running).
PackPool* pack_pool_create() {
  PackPool* p = new (std::nothrow) PackPool;
  if (!p) return nullptr;
  const unsigned hc = std::thread::hardware_concurrency();
  const int nw = std::max(0, std::min(31, (int)(hc ? hc : 2) - 1));  // with the caller: one per core
  try {
    for (int k = 0; k < nw; ++k) p->th.emplace_back([p] { p->loop(); });
  } catch (...) {
    pack_pool_destroy(p);
    return nullptr;
  }
  return p;
}

bool pack_pool_run(PackPool* p, const int8_t* X, int64_t ldx, int n, int ncols, uint8_t* P, int64_t ldp) {
  return p->run(X, ldx, n, ncols, P, ldp);
}

void pack_pool_destroy(PackPool* p) {
  if (!p) return;
  {
    std::lock_guard<std::mutex> lk(p->mu);
    p->quit = true;
  }
  p->cv_go.notify_all();
  for (auto& t : p->th) t.join();
  delete p;
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
  // word k = rows 16g + 4k .. +3: the codes of rows 4k + i (i = 0..3, one per
  // byte k) masked out, then a 4 x 4 byte transpose by byte permutes
  const uint32_t v0 = v & 0x03030303u, v1 = (v >> 2) & 0x03030303u;
  const uint32_t v2 = (v >> 4) & 0x03030303u, v3 = (v >> 6) & 0x03030303u;
  const uint32_t t0 = __byte_perm(v0, v1, 0x5140), t1 = __byte_perm(v2, v3, 0x5140);
  const uint32_t t2 = __byte_perm(v0, v1, 0x7362), t3 = __byte_perm(v2, v3, 0x7362);
  uint32_t w[4] = {__byte_perm(t0, t1, 0x5410), __byte_perm(t0, t1, 0x7632), __byte_perm(t2, t3, 0x5410),
                   __byte_perm(t2, t3, 0x7632)};
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
