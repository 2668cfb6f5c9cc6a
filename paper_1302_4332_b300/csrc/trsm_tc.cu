// a6, split-precision modes: the blocked triangular solve X~ = L^-1 X on the
// 5th-generation tensor cores (tcgen05), operands brought in by TMA,
// accumulators in tensor memory (TMEM).
//
// Same dataflow as the FP64 solve (Sec. 2.2's trsm over a block of SNP
// columns): output tile (k, c) = rows k*TB.., SNP columns c*TN.. is
//     X~_kc = D_k^-1 X_kc + sum_{j<k} (-D_k^-1 L_kj) X~_jc ,
// one product chain with the row panel k of the block operator Aop.
// Precision (the split forms):
//   * Aop is split once at set-up into hi + lo pieces (BF16 or TF32);
//   * the int8 dosages X_kc are exact in BF16/TF32: the diagonal step needs
//     the two products Ahi*X + Alo*X; the cast from int8 happens in shared
//     memory right after the TMA load (no converted copy in HBM);
//   * X~_jc (j < k) are FP32 results of earlier tiles, kept in HBM as hi + lo
//     pieces: three products Ahi*Bhi + Ahi*Blo + Alo*Bhi;
//   * all products accumulate in FP32 in TMEM; the FP32 X~ goes to the
//     FP64 reductions.
//
// Accumulation: the tensor core adds each K-step into its FP32 accumulator
// with truncation, which biases long sums toward zero.  So every 128-wide
// K-block (one j) accumulates into a fresh TMEM partial, and the epilogue
// warps add that partial into an FP32 master held in registers with
// round-to-nearest adds.  Two TMEM partials alternate so the MMAs of block
// j+1 overlap the promotion of block j.
//
// One persistent CTA per SM, 12 warps:
//   warp 0     tile scheduler + TMA producer (one thread)
//   warp 1     MMA issuer (one thread)
//   warps 2-3  int8 -> BF16/TF32 cast of the diagonal block (+ TMEM allocation)
//   warps 4-11 epilogue: warp 4+e owns TMEM lanes 32*(e%4).. and SNP columns
//              128*(e/4)..+127 of the tile; it promotes every partial into
//              its master, then writes FP32 X~ and its hi/lo pieces to HBM
//              and raises the tile's finished-flag (release)
// Operands stream through STAGES shared-memory stages of 64-byte swizzled rows.
// Tiles are handed out in (k, c) order by an atomic counter; a tile waits
// (bounded) on the flag of tile (j, c) before loading X~_jc, so the launch
// cannot deadlock.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cstdio>
#include <cstring>
#include <vector>

#include "tc_ptx.cuh"
#include "trsm_tc.cuh"

namespace gwas {
namespace tc {

constexpr int TN = 256;      // SNP columns per tile (MMA N)
constexpr int STAGES = 4;    // operand stages in shared memory
constexpr int TRING = 2;     // tile-id ring between the scheduler and the other roles
constexpr int EPI_WARPS = 8;
constexpr int THREADS = 32 * (4 + EPI_WARPS);
constexpr int EPI_COLS = TN / 2;  // SNP columns per epilogue warp

template <bool TF32>
struct Cfg {
  static constexpr int ESZ = TF32 ? 4 : 2;       // bytes per operand element
  static constexpr int KCH = 64 / ESZ;           // K per stage: one 64-byte swizzle row
  static constexpr int KMMA = TF32 ? 8 : 16;     // K per tcgen05.mma
  static constexpr int CPB = TB / KCH;           // stages per TB-wide block (4 or 8)
  static constexpr int A_BYTES = TB * 64;        // one piece of A per stage: 8 KB
  static constexpr int B_BYTES = TN * 64;        // one piece of B per stage: 16 KB
  static constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
  static constexpr int X8_BYTES = TN * TB;       // int8 diagonal block: 32 KB
  static constexpr int BAR_OFF = STAGES * STAGE_BYTES + X8_BYTES;
  static constexpr int NBARS = 2 * STAGES + 4 + 2 * TRING + 3;
  static constexpr int SMEM = 1024 + BAR_OFF + NBARS * 8 + TRING * 4 + 16;
};

constexpr int MAX_STUDIES = 8;  // studies in one batched launch

// One study of a launch: its block geometry and buffers.
struct TcStudy {
  int P, C, ncols, n;
  const int8_t* shift;  // per-SNP integer shift c_i (x' = x - c_i on rows < n), or null
  int* flags;           // P x C finished-flags of this launch
  float* xt32;          // FP32 X~ (n_pad x bs); the B "hi" piece in TF32 mode
  void* bhi;            // BF16 mode: hi piece of X~
  void* blo;            // lo piece of X~ (BF16 or FP32)
  int64_t ldt;
};

// The tensor maps of one study: block operator hi/lo, X~ hi/lo, int8 block.
struct TcMaps {
  CUtensorMap Ahi, Alo, Bhi, Blo, X8;
};

// A launch over one or several studies (the batching form): tiles of all
// studies are handed out from one counter in the order of `order`, which
// interleaves the studies row panel by row panel so that every study's
// dependency chain advances while the SMs stay busy.
struct TcBatch {
  TcMaps maps[MAX_STUDIES];
  TcStudy s0;                 // the study when there is only one (order == null)
  const TcStudy* studies;     // device copies of the studies when order != null
  const uint32_t* order;      // tile t -> (study << 28) | (k << 14) | c
  int nstudies, ntiles;
  unsigned int* counter;
  DevStatus* st;
};

__device__ __forceinline__ void decode_tile(const TcBatch& b, int t, int& s, int& k, int& c, TcStudy& S) {
  if (b.order) {
    const uint32_t v = __ldg(b.order + t);
    s = (int)(v >> 28);
    k = (int)((v >> 14) & 0x3FFFu);
    c = (int)(v & 0x3FFFu);
    S = b.studies[s];
  } else {
    S = b.s0;
    s = 0;
    k = t / S.C;
    c = t % S.C;
  }
}

__device__ __forceinline__ uint32_t tf32_trunc_bits(float x) { return __float_as_uint(x) & 0xFFFFE000u; }

template <bool TF32>
__global__ void __launch_bounds__(THREADS, 1)
    trsm_tc_kernel(const __grid_constant__ TcBatch b) {
  using K = Cfg<TF32>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* x8 = smem + STAGES * K::STAGE_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + K::BAR_OFF);
  uint64_t* full = bars;
  uint64_t* empty = full + STAGES;
  uint64_t* part_full = empty + STAGES;
  uint64_t* part_empty = part_full + 2;
  uint64_t* tile_full = part_empty + 2;
  uint64_t* tile_empty = tile_full + TRING;
  uint64_t* x8_full = tile_empty + TRING;
  uint64_t* x8_empty = x8_full + 1;
  uint64_t* drain = x8_empty + 1;
  int* tile_ring = reinterpret_cast<int*>(drain + 1);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tile_ring + TRING);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = b.ntiles;
  DevStatus* st = b.st;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      ptx::mbar_init(&full[s], 2);   // producer (+tx) and producer-or-cast
      ptx::mbar_init(&empty[s], 1);  // MMA commit
    }
    for (int a = 0; a < 2; ++a) {
      ptx::mbar_init(&part_full[a], 1);           // MMA commit
      ptx::mbar_init(&part_empty[a], EPI_WARPS);  // one arrival per epilogue warp
    }
    for (int i = 0; i < TRING; ++i) {
      ptx::mbar_init(&tile_full[i], 1);
      ptx::mbar_init(&tile_empty[i], 1 + 2 + EPI_WARPS);  // MMA + cast warps + epilogue warps
    }
    ptx::mbar_init(x8_full, 1);
    ptx::mbar_init(x8_empty, 1);
    ptx::mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int q = 0; q < b.nstudies; ++q) {
      ptx::prefetch_tensormap(&b.maps[q].Ahi);
      ptx::prefetch_tensormap(&b.maps[q].Alo);
      ptx::prefetch_tensormap(&b.maps[q].Bhi);
      ptx::prefetch_tensormap(&b.maps[q].Blo);
      ptx::prefetch_tensormap(&b.maps[q].X8);
    }
  }
  if (warp == 2) {
    ptx::tmem_alloc(tmem_slot, 2 * TN);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------ scheduler + TMA producer
    if (lane == 0) {
      uint32_t cnt = 0;
      for (int it = 0;; ++it) {
        const int slot = it % TRING;
        const uint32_t use = it / TRING;
        if (!ptx::mbar_wait(&tile_empty[slot], (use & 1) ^ 1, st)) break;
        int t = ptx::aborting(st) ? ntiles : (int)atomicAdd(b.counter, 1u);
        if (t > ntiles) t = ntiles;
        tile_ring[slot] = t;
        ptx::mbar_arrive(&tile_full[slot]);
        if (t >= ntiles) break;
        int sidx, k, c;
        TcStudy S;
        decode_tile(b, t, sidx, k, c, S);
        const TcMaps& M = b.maps[sidx];
        if (!ptx::mbar_wait(x8_empty, (it & 1) ^ 1, st)) break;
        ptx::mbar_arrive_expect_tx(x8_full, K::X8_BYTES);
        ptx::tma_load_2d(x8, &M.X8, x8_full, k * TB, c * TN);
        bool ok = true;
        for (int jj = 0; jj <= k && ok; ++jj) {
          const int j = (jj == 0) ? k : jj - 1;
          if (jj > 0) {
            if (!ptx::wait_flag(&S.flags[j * S.C + c], st)) { ok = false; break; }
            ptx::fence_proxy_async_global();
          }
          for (int h = 0; h < K::CPB; ++h, ++cnt) {
            const int s = cnt % STAGES;
            const uint32_t r = cnt / STAGES;
            if (!ptx::mbar_wait(&empty[s], (r & 1) ^ 1, st)) { ok = false; break; }
            uint8_t* sb = smem + s * K::STAGE_BYTES;
            const int kx = j * TB + h * K::KCH;
            if (jj == 0) {
              ptx::mbar_arrive_expect_tx(&full[s], 2 * K::A_BYTES);
              ptx::tma_load_2d(sb, &M.Ahi, &full[s], kx, k * TB);
              ptx::tma_load_2d(sb + K::A_BYTES, &M.Alo, &full[s], kx, k * TB);
            } else {
              ptx::mbar_arrive_expect_tx(&full[s], 2 * K::A_BYTES + 2 * K::B_BYTES);
              ptx::tma_load_2d(sb, &M.Ahi, &full[s], kx, k * TB);
              ptx::tma_load_2d(sb + K::A_BYTES, &M.Alo, &full[s], kx, k * TB);
              ptx::tma_load_2d(sb + 2 * K::A_BYTES, &M.Bhi, &full[s], kx, c * TN);
              ptx::tma_load_2d(sb + 2 * K::A_BYTES + K::B_BYTES, &M.Blo, &full[s], kx, c * TN);
              ptx::mbar_arrive(&full[s]);
            }
          }
        }
        if (!ok) break;
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = ptx::idesc_f32acc<TF32>(TB, TN);
      uint32_t cnt = 0, kb = 0;
      for (int it = 0;; ++it) {
        const int slot = it % TRING;
        const uint32_t use = it / TRING;
        if (!ptx::mbar_wait(&tile_full[slot], use & 1, st)) break;
        const int t = tile_ring[slot];
        ptx::mbar_arrive(&tile_empty[slot]);
        if (t >= ntiles) break;
        int sidx, k, c;
        TcStudy S;
        decode_tile(b, t, sidx, k, c, S);
        bool ok = true;
        for (int jj = 0; jj <= k && ok; ++jj, ++kb) {
          // a fresh partial per K-block, alternating between the two TMEM buffers
          const int a = kb & 1;
          if (!ptx::mbar_wait(&part_empty[a], ((kb >> 1) & 1) ^ 1, st)) { ok = false; break; }
          ptx::tc_fence_after();
          const uint32_t d = tmem_base + a * TN;
          uint32_t accumulate = 0;
          for (int h = 0; h < K::CPB; ++h, ++cnt) {
            const int s = cnt % STAGES;
            const uint32_t r = cnt / STAGES;
            if (!ptx::mbar_wait(&full[s], r & 1, st)) { ok = false; break; }
            ptx::tc_fence_after();
            const uint32_t base = ptx::smem_u32(smem + s * K::STAGE_BYTES);
#pragma unroll
            for (int kk = 0; kk < K::KCH / K::KMMA; ++kk) {
              const uint32_t off = kk * K::KMMA * K::ESZ;
              const uint64_t ahi = ptx::sdesc_k64(base + off);
              const uint64_t alo = ptx::sdesc_k64(base + K::A_BYTES + off);
              const uint64_t bhi = ptx::sdesc_k64(base + 2 * K::A_BYTES + off);
              const uint64_t blo = ptx::sdesc_k64(base + 2 * K::A_BYTES + K::B_BYTES + off);
              ptx::mma<TF32>(d, alo, bhi, idesc, accumulate);
              accumulate = 1;
              if (jj > 0) ptx::mma<TF32>(d, ahi, blo, idesc, 1);
              ptx::mma<TF32>(d, ahi, bhi, idesc, 1);
            }
            ptx::mma_commit(&empty[s]);
          }
          if (!ok) break;
          ptx::mma_commit(&part_full[a]);
        }
        if (!ok) break;
      }
    }
  } else if (warp < 4) {
    // ---------------------------------------- int8 -> BF16/TF32 cast (diagonal block)
    // The 64 threads decide together (group_and) after every wait.
    const int ct = threadIdx.x - 64;  // 0..63
    constexpr int E = 16 / K::ESZ;    // elements per 16-byte chunk
    uint32_t cnt = 0;
    for (int it = 0;; ++it) {
      const int slot = it % TRING;
      const uint32_t use = it / TRING;
      if (!ptx::group_and(2, 64, ptx::mbar_wait(&tile_full[slot], use & 1, st))) break;
      const int t = tile_ring[slot];
      ptx::named_bar(2, 64);
      if (lane == 0) ptx::mbar_arrive(&tile_empty[slot]);
      if (t >= ntiles) break;
      int sidx, k, ctile;
      TcStudy S;
      decode_tile(b, t, sidx, k, ctile, S);
      if (!ptx::group_and(2, 64, ptx::mbar_wait(x8_full, it & 1, st))) break;
      bool ok = true;
      for (int h = 0; h < K::CPB; ++h) {
        const int s = (cnt + h) % STAGES;
        const uint32_t r = (cnt + h) / STAGES;
        if (!ptx::group_and(2, 64, ptx::mbar_wait(&empty[s], (r & 1) ^ 1, st))) { ok = false; break; }
        uint8_t* bh = smem + s * K::STAGE_BYTES + 2 * K::A_BYTES;
        for (int col = ct; col < TN; col += 64) {
          const int8_t* src = reinterpret_cast<const int8_t*>(x8 + col * TB + h * K::KCH);
          const int colg = ctile * TN + col;
          const int csh = (S.shift && colg < S.ncols) ? S.shift[colg] : 0;
          const int row0 = k * TB + h * K::KCH;
#pragma unroll
          for (int q = 0; q < 4; ++q) {  // four 16-byte chunks per 64-byte row
            // x' = x - c on the n sample rows, 0 on the padding (exact small integers)
            float f[E];
            if constexpr (TF32) {
              const char4 v = *reinterpret_cast<const char4*>(src + q * E);
              const signed char e4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
              for (int i = 0; i < 4; ++i) f[i] = (row0 + q * E + i < S.n) ? (float)(e4[i] - csh) : 0.f;
            } else {
              const char4 v0 = *reinterpret_cast<const char4*>(src + q * E);
              const char4 v1 = *reinterpret_cast<const char4*>(src + q * E + 4);
              const signed char e8[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
              for (int i = 0; i < 8; ++i) f[i] = (row0 + q * E + i < S.n) ? (float)(e8[i] - csh) : 0.f;
            }
            uint32_t w[4];
            if constexpr (TF32) {
#pragma unroll
              for (int i = 0; i < 4; ++i) w[i] = __float_as_uint(f[i]);
            } else {
#pragma unroll
              for (int i = 0; i < 4; ++i) {
                const __nv_bfloat162 b2 = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
                w[i] = *reinterpret_cast<const uint32_t*>(&b2);
              }
            }
            // 64-byte swizzle: 16-byte chunk q of row col sits at chunk q ^ ((col >> 1) & 3)
            *reinterpret_cast<uint4*>(bh + col * 64 + ((q ^ ((col >> 1) & 3)) << 4)) =
                make_uint4(w[0], w[1], w[2], w[3]);
          }
        }
        ptx::fence_proxy_async_shared();
        ptx::named_bar(2, 64);
        if (ct == 0) ptx::mbar_arrive(&full[s]);
      }
      if (!ok) break;
      if (ct == 0) ptx::mbar_arrive(x8_empty);
      cnt += K::CPB * (k + 1);
    }
  } else {
    // ----------------------------------------------------------------- epilogue
    // The EPI_WARPS warps decide together (group_and) after every wait.
    constexpr int NT = 32 * EPI_WARPS;
    const int e = warp - 4;
    const int lq = e & 3;           // TMEM lanes 32 lq .. 32 lq + 31
    const int chalf = e >> 2;       // SNP columns chalf * EPI_COLS ..
    uint32_t kb = 0;
    float master[EPI_COLS];
    for (int it = 0;; ++it) {
      const int slot = it % TRING;
      const uint32_t use = it / TRING;
      if (!ptx::group_and(1, NT, ptx::mbar_wait(&tile_full[slot], use & 1, st))) break;
      const int t = tile_ring[slot];
      ptx::named_bar(1, NT);
      if (lane == 0) ptx::mbar_arrive(&tile_empty[slot]);
      if (t >= ntiles) break;
      int sidx, k, c;
      TcStudy S;
      decode_tile(b, t, sidx, k, c, S);
#pragma unroll
      for (int i = 0; i < EPI_COLS; ++i) master[i] = 0.f;
      bool ok = true;
      for (int jj = 0; jj <= k; ++jj, ++kb) {
        const int a = kb & 1;
        if (!ptx::group_and(1, NT, ptx::mbar_wait(&part_full[a], (kb >> 1) & 1, st))) { ok = false; break; }
        ptx::tc_fence_after();
        const uint32_t tb = tmem_base + (static_cast<uint32_t>(32 * lq) << 16) + a * TN + chalf * EPI_COLS;
#pragma unroll
        for (int ch = 0; ch < EPI_COLS / 16; ++ch) {
          uint32_t v[16];
          ptx::tmem_ld_32x32b_x16(tb + ch * 16, v);
          ptx::tmem_ld_wait();
#pragma unroll
          for (int i = 0; i < 16; ++i) master[ch * 16 + i] += __uint_as_float(v[i]);  // round to nearest
        }
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&part_empty[a]);
      }
      if (!ok) break;
      const int64_t row = (int64_t)k * TB + 32 * lq + lane;
      const int col0 = c * TN + chalf * EPI_COLS;
#pragma unroll
      for (int i = 0; i < EPI_COLS; ++i) {
        const int col = col0 + i;
        if (col < S.ncols) {
          const float x = master[i];
          const int64_t idx = (int64_t)col * S.ldt + row;
          S.xt32[idx] = x;
          if constexpr (TF32) {
            static_cast<float*>(S.blo)[idx] = x - __uint_as_float(tf32_trunc_bits(x));
          } else {
            const __nv_bfloat16 hi = __float2bfloat16_rn(x);
            static_cast<__nv_bfloat16*>(S.bhi)[idx] = hi;
            static_cast<__nv_bfloat16*>(S.blo)[idx] = __float2bfloat16_rn(x - __bfloat162float(hi));
          }
        }
      }
      ptx::named_bar(1, NT);
      if (e == 0 && lane == 0) {
        ptx::fence_proxy_async_global();
        __threadfence();
        ptx::st_release(&S.flags[k * S.C + c], 1);
      }
    }
  }

  // ---------------------------------------------------------------- teardown
  if (warp == 1 && lane == 0) {
    // every MMA this CTA issued has completed before TMEM is released
    ptx::mma_commit(drain);
    const long long t0 = ptx::globaltimer();
    while (!ptx::mbar_try_wait(drain, 0) && ptx::globaltimer() - t0 < 100000000LL) {
    }
  }
  if (ptx::aborting(st)) {
    // an aborted launch may still have TMA copies in flight into this CTA's
    // shared memory: give them time to land before the CTA retires
    const long long t0 = ptx::globaltimer();
    while (ptx::globaltimer() - t0 < 2000000LL) {
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  if (warp == 2) ptx::tmem_dealloc(tmem_base, 2 * TN);
}

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

// ------------------------------------------------------------ set-up kernels
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
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

struct TcState {
  bool tf32 = false;
  int n = 0, n_pad = 0, bs = 0, P = 0, num_sms = 0;
  void* ahi = nullptr;
  void* alo = nullptr;
  float* xt32 = nullptr;
  void* bhi = nullptr;
  void* blo = nullptr;
  int64_t ldt = 0;
  int8_t* shift = nullptr;        // per-SNP integer shift (bs)
  bool center = false;            // X_L[:, 0] is the intercept: shift SNP columns
  int strip_group = 0;            // tile order over groups of column strips (0: all)
  uint32_t* order = nullptr;      // device tile order when strip_group > 0
  TcStudy* study_dev = nullptr;   // device copy of the study descriptor (grouped order)
  int order_C = -1;               // the column-strip count the order was built for
  unsigned int* sched = nullptr;  // [0] counter, flags from +32
  size_t sched_bytes = 0;
  DevStatus* st = nullptr;
  CUtensorMap mAhi, mAlo, mBhi, mBlo;
  EncodeTiledFn encode = nullptr;
};

static cudaError_t get_encode(EncodeTiledFn* fn) {
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
static cudaError_t make_map(EncodeTiledFn enc, CUtensorMap* m, CUtensorMapDataType dt, const void* base,
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

template <bool TF32>
static cudaError_t set_smem_attr() {
  return cudaFuncSetAttribute(trsm_tc_kernel<TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<TF32>::SMEM);
}

cudaError_t create(TcState** out, Split split, const double* Aop, int n, int n_pad, int bs, int num_sms,
                   bool center, DevStatus* st, cudaStream_t s, int64_t* launches, int strip_group) {
  *out = nullptr;
  TcState* t = new TcState;
  t->tf32 = (split == SPLIT_TF32);
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
  TRY(cudaMalloc(&t->shift, (size_t)bs));
  t->center = center;
  t->strip_group = strip_group;
  if (strip_group > 0) {
    TRY(cudaMalloc(&t->order, sizeof(uint32_t) * (size_t)t->P * Cmax));
    TRY(cudaMalloc(&t->study_dev, sizeof(TcStudy)));
  }
  t->sched_bytes = 128 + sizeof(int) * (size_t)t->P * Cmax;
  TRY(cudaMalloc(&t->sched, t->sched_bytes));
  TRY(cudaMemsetAsync(t->sched, 0, t->sched_bytes, s));
  if (t->tf32)
    split_aop_kernel<true><<<1184, 256, 0, s>>>(Aop, (int64_t)n2, t->ahi, t->alo);
  else
    split_aop_kernel<false><<<1184, 256, 0, s>>>(Aop, (int64_t)n2, t->ahi, t->alo);
  ++*launches;
  TRY(cudaGetLastError());
  const CUtensorMapDataType dt = t->tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const uint32_t kch = t->tf32 ? Cfg<true>::KCH : Cfg<false>::KCH;
  TRY(make_map(t->encode, &t->mAhi, dt, t->ahi, n_pad, n_pad, esz * n_pad, kch, TB, true));
  TRY(make_map(t->encode, &t->mAlo, dt, t->alo, n_pad, n_pad, esz * n_pad, kch, TB, true));
  const void* bhi_base = t->tf32 ? static_cast<const void*>(t->xt32) : t->bhi;
  TRY(make_map(t->encode, &t->mBhi, dt, bhi_base, n_pad, bs, esz * n_pad, kch, TN, true));
  TRY(make_map(t->encode, &t->mBlo, dt, t->blo, n_pad, bs, esz * n_pad, kch, TN, true));
  TRY(t->tf32 ? set_smem_attr<true>() : set_smem_attr<false>());
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

// The study part of one launch: int8 map, cleared flags, integer shifts.
static cudaError_t prepare_study(TcState* t, const int8_t* X, int64_t ldx, int ncols, cudaStream_t s,
                                 int64_t* launches, TcStudy* S, CUtensorMap* mX8) {
  if (ncols > t->bs || (reinterpret_cast<uintptr_t>(X) & 15) || (ldx & 15) || ldx < t->n)
    return cudaErrorInvalidValue;
  cudaError_t e = make_map(t->encode, mX8, CU_TENSOR_MAP_DATA_TYPE_UINT8, X, (uint64_t)t->n, (uint64_t)ncols,
                           (uint64_t)ldx, TB, TN, false);
  if (e != cudaSuccess) return e;
  const int C = (ncols + TN - 1) / TN;
  e = cudaMemsetAsync(t->sched, 0, 128 + sizeof(int) * (size_t)t->P * C, s);
  if (e != cudaSuccess) return e;
  if (t->center) {
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
  return cudaSuccess;
}

static cudaError_t launch_kernel(bool tf32, const TcBatch& b, int num_sms, cudaStream_t s, int64_t* launches) {
  const int grid = b.ntiles < num_sms ? b.ntiles : num_sms;
  if (tf32)
    trsm_tc_kernel<true><<<grid, THREADS, Cfg<true>::SMEM, s>>>(b);
  else
    trsm_tc_kernel<false><<<grid, THREADS, Cfg<false>::SMEM, s>>>(b);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t run_block(TcState* t, const int8_t* X, int64_t ldx, int ncols, cudaStream_t s, int64_t* launches) {
  if (ncols <= 0) return cudaSuccess;
  TcBatch b;
  memset(&b, 0, sizeof b);
  cudaError_t e = prepare_study(t, X, ldx, ncols, s, launches, &b.s0, &b.maps[0].X8);
  if (e != cudaSuccess) return e;
  b.maps[0].Ahi = t->mAhi;
  b.maps[0].Alo = t->mAlo;
  b.maps[0].Bhi = t->mBhi;
  b.maps[0].Blo = t->mBlo;
  b.nstudies = 1;
  b.ntiles = t->P * b.s0.C;
  b.counter = t->sched;
  b.st = t->st;
  if (t->strip_group > 0 && t->strip_group < b.s0.C) {
    if (t->order_C != b.s0.C) {  // (re)build the grouped order for this strip count
      std::vector<uint32_t> order;
      append_study_order(order, 0, t->P, b.s0.C, t->strip_group);
      if ((e = cudaMemcpyAsync(t->order, order.data(), sizeof(uint32_t) * order.size(), cudaMemcpyHostToDevice, s)) !=
              cudaSuccess ||
          (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return e;
      t->order_C = b.s0.C;
    }
    // the grouped order reads the study descriptor from device memory
    if ((e = cudaMemcpyAsync(t->study_dev, &b.s0, sizeof(TcStudy), cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
    b.order = t->order;
    b.studies = t->study_dev;
  }
  return launch_kernel(t->tf32, b, t->num_sms, s, launches);
}

// ------------------------------------------------------------- batched launch
struct TcBatchState {
  int nstudies = 0;
  int ntiles = 0;
  TcStudy S[MAX_STUDIES];
  CUtensorMap mX8[MAX_STUDIES];
  const int8_t* X[MAX_STUDIES];
  int64_t ldx[MAX_STUDIES];
  bool tf32 = false;
  int num_sms = 0;
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
    if (ts[i]->tf32 != ts[0]->tf32) return cudaErrorInvalidValue;
  TcBatchState* B = new TcBatchState;
  B->nstudies = nstudies;
  B->tf32 = ts[0]->tf32;
  B->num_sms = ts[0]->num_sms;
  B->st = ts[0]->st;
  size_t cap = 0;
  for (int i = 0; i < nstudies; ++i) cap += (size_t)ts[i]->P * ((ts[i]->bs + TN - 1) / TN);
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
    pmax = t->P > pmax ? t->P : pmax;
    total += S[i].P * S[i].C;
  }
  std::vector<uint32_t> order;
  order.reserve(total);
  if (order_mode == 0) {
    for (int k = 0; k < pmax; ++k)
      for (int i = 0; i < B->nstudies; ++i)
        if (ncols[i] > 0 && k < S[i].P)
          for (int c = 0; c < S[i].C; ++c) order.push_back(((uint32_t)i << 28) | ((uint32_t)k << 14) | (uint32_t)c);
  } else {
    for (int i = 0; i < B->nstudies; ++i)
      if (ncols[i] > 0) append_study_order(order, i, S[i].P, S[i].C, strip_group);
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
  for (int i = 0; i < B->nstudies; ++i) {
    if (B->S[i].ncols == 0) continue;
    TcState* t = ts[i];
    if ((e = cudaMemsetAsync(t->sched, 0, 128 + sizeof(int) * (size_t)t->P * B->S[i].C, s)) != cudaSuccess) return e;
    if (t->center) {
      column_shift_kernel<<<(B->S[i].ncols + 7) / 8, 256, 0, s>>>(B->X[i], B->ldx[i], t->n, B->S[i].ncols, t->shift);
      ++*launches;
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    b.maps[i].Ahi = t->mAhi;
    b.maps[i].Alo = t->mAlo;
    b.maps[i].Bhi = t->mBhi;
    b.maps[i].Blo = t->mBlo;
    b.maps[i].X8 = B->mX8[i];
  }
  if ((e = cudaMemsetAsync(B->d_counter, 0, 128, s)) != cudaSuccess) return e;
  b.studies = B->d_studies;
  b.order = B->d_order;
  b.nstudies = B->nstudies;
  b.ntiles = B->ntiles;
  b.counter = B->d_counter;
  b.st = B->st;
  return launch_kernel(B->tf32, b, B->num_sms, s, launches);
}

void batch_destroy(TcBatchState* B) {
  if (!B) return;
  cudaFree(B->d_studies);
  cudaFree(B->d_order);
  cudaFree(B->d_counter);
  delete B;
}

const float* xt_f32(const TcState* t) { return t->xt32; }
const int8_t* shift_of(const TcState* t) { return t->center ? t->shift : nullptr; }
int64_t xt_ld(const TcState* t) { return t->ldt; }

void destroy(TcState* t) {
  if (!t) return;
  cudaFree(t->ahi);
  cudaFree(t->alo);
  cudaFree(t->xt32);
  cudaFree(t->bhi);
  cudaFree(t->blo);
  cudaFree(t->sched);
  cudaFree(t->shift);
  cudaFree(t->order);
  cudaFree(t->study_dev);
  delete t;
}

}  // namespace tc
}  // namespace gwas
