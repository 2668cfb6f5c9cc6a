// a6, split-precision modes: the blocked triangular solve X~ = L^-1 X on the
// 5th-generation tensor cores (tcgen05), operands brought in by TMA,
// accumulators in tensor memory (TMEM).  This file holds the solve kernels --
// the substitution (single CTAs, pair product) and the
// inverse form (the product with a precomputed L^-1, further below) -- and
// their launch entries; per-study state, set-up and pre-passes are in
// trsm_tc_host.cu.
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
// K-block accumulates into a fresh TMEM
// partial, and the epilogue warps add that partial into an FP32 master held
// in registers with round-to-nearest adds.  Two TMEM partials alternate so
// the MMAs of the next blocks overlap the promotion of the last ones.
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

#include <cstring>

#include "tc_ptx.cuh"
#include "trsm_tc_kernels.cuh"

namespace gwas {
namespace tc {

__device__ __forceinline__ void decode_tile(const TcBatch& b, int t, int& s, int& k, int& c, TcStudy& S) {
  if (b.order) {
    const uint32_t v = __ldg(b.order + t);
    s = (int)(v >> 28);
    k = (int)((v >> 14) & 0x3FFFu);
    c = (int)(v & 0x3FFFu);
    S = b.studies ? b.studies[s] : b.s0;  // one study: its descriptor travels in the launch parameters
  } else {
    S = b.s0;
    s = 0;
    k = t / S.C;
    c = t % S.C;
  }
}

__device__ __forceinline__ uint32_t tf32_trunc_bits(float x) { return __float_as_uint(x) & 0xFFFFE000u; }

// Epilogue stores of one warp's 32 rows x EPI_COLS columns of X~: the FP32
// value (for the reductions; in TF32 mode also the hi operand) and the lo
// piece, plus the BF16 hi piece in BF16 mode.
template <bool TF32>
__device__ __forceinline__ void store_tile(const float (&master)[EPI_COLS], const TcStudy& S, int64_t xrow,
                                           int col0) {
#pragma unroll
  for (int i = 0; i < EPI_COLS; ++i) {
    const int col = col0 + i;
    if (col < S.ncols) {
      const float x = master[i];
      const int64_t idx = (int64_t)col * S.ldt + xrow;
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
}

// K-block kinds of a work unit's stage sequence.
enum KbKind : int {
  KB_DIAG = 0,    // j == k: Aop hi/lo by TMA, B = the int8 block cast in shared memory
  KB_LOCAL = 2    // Aop and all of X~_jc by this CTA
};

// A work unit: the tile (k, c).
struct Unit {
  int k;    // row panel
  int nkb;  // K-blocks in the unit's stage sequence
};

__device__ __forceinline__ Unit make_unit(int row) {
  Unit u;
  u.k = row;
  u.nkb = row + 1;
  return u;
}

// K-block jj of a unit: its kind, and j, the block column of Aop it multiplies
// (forward: the diagonal block first, then 0 .. k-1).
__device__ __forceinline__ KbKind kb_kind(const Unit& u, int jj, int& j) {
  if (jj == 0) {
    j = u.k;
    return KB_DIAG;
  }
  j = jj - 1;
  return KB_LOCAL;
}

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
  uint64_t* peer_free = drain + 1;  // unused (kept so the barrier block keeps its size)
  int* tile_ring = reinterpret_cast<int*>(peer_free + TRING);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tile_ring + TRING);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = b.ntiles;  // work units
  DevStatus* st = b.st;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      ptx::mbar_init(&full[s], 2);   // producer (+tx) and producer-or-cast
      ptx::mbar_init(&empty[s], 1);  // the MMA commit
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
      uint32_t cnt = 0, x8n = 0;
      for (int it = 0;; ++it) {
        const int slot = it % TRING;
        const uint32_t use = it / TRING;
        if (!ptx::mbar_wait(&tile_empty[slot], (use & 1) ^ 1, st)) break;
        int t = ptx::aborting(st) ? ntiles : (int)atomicAdd(b.counter, 1u);
        if (t > ntiles) t = ntiles;
        tile_ring[slot] = t;
        ptx::mbar_arrive(&tile_full[slot]);
        if (t >= ntiles) break;
        int sidx, row, c;
        TcStudy S;
        decode_tile(b, t, sidx, row, c, S);
        const TcMaps& M = b.maps[sidx];
        const Unit u = make_unit(row);
        {
          if (!ptx::mbar_wait(x8_empty, (x8n & 1) ^ 1, st)) break;
          ptx::mbar_arrive_expect_tx(x8_full, K::X8_BYTES);
          ptx::tma_load_2d(x8, &M.X8, x8_full, u.k * TB, c * TN);
          ++x8n;
        }
        bool ok = true;
        for (int jj = 0; jj < u.nkb && ok; ++jj) {
          int j;
          const KbKind kind = kb_kind(u, jj, j);
          if (kind == KB_LOCAL) {
            if (!ptx::wait_flag(&S.flags[j * S.C + c], st)) { ok = false; break; }
            ptx::fence_proxy_async_global();
          }
          for (int h = 0; h < K::CPB; ++h, ++cnt) {
            const int s = cnt % STAGES;
            const uint32_t r = cnt / STAGES;
            if (!ptx::mbar_wait(&empty[s], (r & 1) ^ 1, st)) { ok = false; break; }
            uint8_t* sb = smem + s * K::STAGE_BYTES;
            const int kx = j * TB + h * K::KCH;
            if (kind == KB_DIAG) {
              ptx::mbar_arrive_expect_tx(&full[s], 2 * K::A_BYTES);
              ptx::tma_load_2d(sb, &M.Ahi, &full[s], kx, u.k * TB);
              ptx::tma_load_2d(sb + K::A_BYTES, &M.Alo, &full[s], kx, u.k * TB);
            } else {
              ptx::mbar_arrive_expect_tx(&full[s], 2 * K::A_BYTES + 2 * K::B_BYTES);
              ptx::tma_load_2d(sb, &M.Ahi, &full[s], kx, u.k * TB);
              ptx::tma_load_2d(sb + K::A_BYTES, &M.Alo, &full[s], kx, u.k * TB);
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
      auto release = [&](int s) { ptx::mma_commit(&empty[s]); };  // a consumed stage goes back to the producer
      for (int it = 0;; ++it) {
        const int slot = it % TRING;
        const uint32_t use = it / TRING;
        if (!ptx::mbar_wait(&tile_full[slot], use & 1, st)) break;
        const int t = tile_ring[slot];
        ptx::mbar_arrive(&tile_empty[slot]);
        if (t >= ntiles) break;
        int sidx, row, c;
        TcStudy S;
        decode_tile(b, t, sidx, row, c, S);
        const Unit u = make_unit(row);
        bool ok = true;
        int q = 0;  // K-blocks of the tile issued so far
        int a = 0;
        uint32_t d = 0, accumulate = 0;
        for (int jj = 0; jj < u.nkb && ok; ++jj) {
          int j;
          const KbKind kind = kb_kind(u, jj, j);
          if (q % PROMOTE == 0) {
            // a fresh partial every PROMOTE K-blocks, alternating between the two TMEM buffers
            a = kb & 1;
            if (!ptx::mbar_wait(&part_empty[a], ((kb >> 1) & 1) ^ 1, st)) { ok = false; break; }
            ++kb;
            ptx::tc_fence_after();
            d = tmem_base + a * TN;
            accumulate = 0;
          }
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
              if (kind != KB_DIAG) ptx::mma<TF32>(d, ahi, blo, idesc, 1);
              ptx::mma<TF32>(d, ahi, bhi, idesc, 1);
            }
            release(s);
          }
          if (!ok) break;
          const int nk = u.k + 1;  // the tile's K-blocks
          if (q % PROMOTE == PROMOTE - 1 || q == nk - 1) ptx::mma_commit(&part_full[a]);
          ++q;
        }
        if (!ok) break;
      }
    }
  } else if (warp < 4) {
    // ---------------------------------------- int8 -> BF16/TF32 cast (diagonal block)
    // The 64 threads decide together (group_and) after every wait.
    const int ct = threadIdx.x - 64;  // 0..63
    constexpr int E = 16 / K::ESZ;    // elements per 16-byte chunk
    uint32_t cnt = 0, x8n = 0;
    for (int it = 0;; ++it) {
      const int slot = it % TRING;
      const uint32_t use = it / TRING;
      if (!ptx::group_and(2, 64, ptx::mbar_wait(&tile_full[slot], use & 1, st))) break;
      const int t = tile_ring[slot];
      ptx::named_bar(2, 64);
      if (lane == 0) ptx::mbar_arrive(&tile_empty[slot]);
      if (t >= ntiles) break;
      int sidx, row, ctile;
      TcStudy S;
      decode_tile(b, t, sidx, row, ctile, S);
      const Unit u = make_unit(row);
      {
        const int k = u.k;
        if (!ptx::group_and(2, 64, ptx::mbar_wait(x8_full, x8n & 1, st))) break;
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
        ++x8n;
      }
      cnt += K::CPB * u.nkb;
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
      int sidx, row, c;
      TcStudy S;
      decode_tile(b, t, sidx, row, c, S);
      const Unit u = make_unit(row);
      const int k = u.k;
#pragma unroll
      for (int i = 0; i < EPI_COLS; ++i) master[i] = 0.f;
      bool ok = true;
      const int nk = k + 1;  // the tile's K-blocks
      const int npart = (nk + PROMOTE - 1) / PROMOTE;
      for (int jp = 0; jp < npart; ++jp, ++kb) {
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
      const int64_t xrow = (int64_t)k * TB + 32 * lq + lane;
      const int col0 = c * TN + chalf * EPI_COLS;
      store_tile<TF32>(master, S, xrow, col0);
      ptx::named_bar(1, NT);
      ptx::publish_flag(&S.flags[k * S.C + c], e == 0 && lane == 0);
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

// ---------------------------------------------------------------------------
// Pair-MMA mode: the row panels 2u and 2u+1 of a strip as one M = 256 product
// on the two SMs of a cluster (tcgen05 cta_group::2).  CTA r holds the block
// operator rows of panel 2u + r and SNP columns r*128.. of the strip's X~
// blocks; the pair's tensor cores share the two B halves, so each CTA lands
// 128 KB per K-block (not 192 KB).  The operator's odd row panels are the
// pair form A' (built at set-up, pair_rows_kernel): panel 2u+1 re-expressed
// through panel 2u's own equation, so that neither row of a pair needs the
// other's result (the blocked solve with 256-row diagonal blocks):
//   D0   A = [A_{2u,2u} ; A'_{2u+1,2u}],   B = X_{2u}    (int8, cast in shared memory)
//   D1   A = [0 ; A_{2u+1,2u+1}],          B = X_{2u+1}  (int8; a TMA box wholly
//                                                          outside the operator reads zeros)
//   M_j  A = [A_{2u,j} ; A'_{2u+1,j}],     B = X~_j,  j < 2u
// all into the shared partials.  The last unit of an odd P has panel 2u
// only: D0 and the M_j with CTA 1's A rows zero.  CTA 0 issues every MMA;
// both CTAs' loads and casts complete on CTA 0's stage barriers, and CTA 0's
// commits release both CTAs' stages and partials.
namespace pair2 {
constexpr int STAGES = 5;

template <bool TF32>
struct Cfg {
  static constexpr int ESZ = TF32 ? 4 : 2;
  static constexpr int KCH = 64 / ESZ;
  static constexpr int KMMA = TF32 ? 8 : 16;
  static constexpr int CPB = TB / KCH;
  static constexpr int A_BYTES = TB * 64;                        // one piece of this CTA's A rows: 8 KB
  static constexpr int B_BYTES = (TN / 2) * 64;                  // one piece of this CTA's B half: 8 KB
  static constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;  // 32 KB
  static constexpr int X8H_BYTES = (TN / 2) * TB;                // int8 block, this CTA's columns: 16 KB
  // epilogue staging, per warp two 2 KB chunk buffers (32 rows x st_cols())
  static constexpr int CHUNK_BYTES = 2048;
  static constexpr int STG_OFF = STAGES * STAGE_BYTES + 2 * X8H_BYTES;
  static constexpr int BAR_OFF = STG_OFF + EPI_WARPS * 2 * CHUNK_BYTES;
  static constexpr int NBARS = 2 * STAGES + 4 + 3 * TRING + 3;
  static constexpr int SMEM = 1024 + BAR_OFF + NBARS * 8 + TRING * 4 + 16;
};

enum Kind : int { D0 = 0, D1 = 1, MJ = 2 };

struct Unit {
  int k0;       // panel 2u (CTA 0); CTA 1 has panel k0 + 1 when paired
  bool paired;  // panel k0 + 1 exists
  int nkb;      // K-blocks, all into the shared partials
};

__device__ __forceinline__ Unit make_unit(int row, const TcStudy& S) {
  Unit u;
  u.k0 = 2 * row;
  u.paired = u.k0 + 1 < S.P;
  u.nkb = u.k0 + (u.paired ? 2 : 1);
  return u;
}

// The inverse form pairs panels (2u - o, 2u + 1 - o) with o = P mod 2: with an
// odd panel count the lone panel is panel 0 (one K-block, the partner CTA's
// half of its one MMA on zero rows) instead of the last one (P K-blocks).  The
// substitution keeps pairs (2u, 2u + 1): its operator's pair form is built on them.
__device__ __forceinline__ Unit make_unit_inv(int row, const TcStudy& S) {
  Unit u;
  const int o = S.P & 1;
  if (o && row == 0) {
    u.k0 = 0;
    u.paired = false;
    u.nkb = 1;
    return u;
  }
  u.k0 = 2 * row - o;
  u.paired = u.k0 + 1 < S.P;
  u.nkb = u.k0 + (u.paired ? 2 : 1);
  return u;
}

// K-block jj of a unit: its kind, the operator block column j, and the
// operator row panel of this CTA's A rows (-1: zero rows).
__device__ __forceinline__ Kind kind_of(const Unit& u, uint32_t rank, int jj, int& j, int& arow) {
  const int k1 = u.k0 + 1;
  if (jj == 0) {
    j = u.k0;
    arow = rank == 0 ? u.k0 : (u.paired ? k1 : -1);
    return D0;
  }
  if (u.paired && jj == 1) {
    j = k1;
    arow = rank == 1 ? k1 : -1;
    return D1;
  }
  j = jj - (u.paired ? 2 : 1);
  arow = rank == 0 ? u.k0 : (u.paired ? k1 : -1);
  return MJ;
}
}  // namespace pair2

template <bool TF32>
__global__ void __launch_bounds__(THREADS, 1)
    trsm_tc_pair_mma_kernel(const __grid_constant__ TcBatch b) {
  using K = pair2::Cfg<TF32>;
  constexpr int ST = pair2::STAGES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* x8 = smem + ST * K::STAGE_BYTES;  // int8 blocks of panels 2u, 2u+1 (this CTA's columns)
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + K::BAR_OFF);
  uint64_t* full = bars;               // CTA 0: both CTAs' loads and casts of a stage
  uint64_t* empty = full + ST;         // CTA 0's commit: the stage's MMAs are done
  uint64_t* part_full = empty + ST;    // CTA 0's commit: a partial is complete
  uint64_t* part_empty = part_full + 2;  // CTA 0: both CTAs' epilogues are done with a partial
  uint64_t* tile_full = part_empty + 2;
  uint64_t* tile_empty = tile_full + TRING;
  uint64_t* x8_full = tile_empty + TRING;
  uint64_t* x8_empty = x8_full + 1;
  uint64_t* drain = x8_empty + 1;
  uint64_t* peer_free = drain + 1;
  int* tile_ring = reinterpret_cast<int*>(peer_free + TRING);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tile_ring + TRING);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = b.ntiles;  // work units: row-panel pairs of a strip
  DevStatus* st = b.st;
  const uint32_t rank = ptx::cluster_ctarank();
  const bool leader = rank == 0;
  constexpr uint16_t BOTH = 3;
  // a barrier of CTA 0, as this CTA addresses it
  auto lead_addr = [&](uint64_t* bar) -> uint32_t { return leader ? ptx::smem_u32(bar) : ptx::peer_addr(bar, 0); };
  // counting arrival on a barrier of CTA 0 (no data of this thread to publish)
  auto count_lead = [&](uint64_t* bar) {
    if (leader)
      ptx::mbar_arrive(bar);
    else
      ptx::mbar_arrive_peer_count(ptx::peer_addr(bar, 0));
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) {
      ptx::mbar_init(&full[s], 4);   // two arrivals from each CTA (+ the bytes of both)
      ptx::mbar_init(&empty[s], 1);  // CTA 0's commit
    }
    for (int a = 0; a < 2; ++a) {
      ptx::mbar_init(&part_full[a], 1);
      ptx::mbar_init(&part_empty[a], 2 * EPI_WARPS);
    }
    for (int i = 0; i < TRING; ++i) {
      ptx::mbar_init(&tile_full[i], 1);
      ptx::mbar_init(&tile_empty[i], 1 + 2 + EPI_WARPS);
      ptx::mbar_init(&peer_free[i], 1);
    }
    ptx::mbar_init(x8_full, 1);
    ptx::mbar_init(x8_empty, 1);
    ptx::mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int q = 0; q < b.nstudies; ++q) {
      ptx::prefetch_tensormap(&b.maps[q].Ahi);
      ptx::prefetch_tensormap(&b.maps[q].Alo);
      ptx::prefetch_tensormap(&b.maps[q].BhiH);
      ptx::prefetch_tensormap(&b.maps[q].BloH);
      ptx::prefetch_tensormap(&b.maps[q].X8H);
    }
  }
  if (warp == 2) {
    ptx::tmem_alloc_pair(tmem_slot, 2 * TN);
    ptx::tmem_relinquish_pair();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  ptx::cluster_sync();  // both CTAs' barriers and tensor memory exist before any remote access
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------ scheduler + TMA producer
    if (lane == 0) {
      uint32_t cnt = 0, x8n = 0;
      for (int it = 0;; ++it) {
        const int slot = it % TRING;
        const uint32_t use = it / TRING;
        if (!ptx::mbar_wait(&tile_empty[slot], (use & 1) ^ 1, st)) break;
        int t;
        if (leader) {
          if (!ptx::mbar_wait(&peer_free[slot], use & 1, st)) break;
          t = ptx::aborting(st) ? ntiles : (int)atomicAdd(b.counter, 1u);
          if (t > ntiles) t = ntiles;
          tile_ring[slot] = t;
          ptx::st_peer_u32(ptx::peer_addr(&tile_ring[slot], 1), (uint32_t)t);
          ptx::mbar_arrive(&tile_full[slot]);
          ptx::mbar_arrive_peer(ptx::peer_addr(&tile_full[slot], 1));
        } else {
          ptx::mbar_arrive_peer(ptx::peer_addr(&peer_free[slot], 0));
          if (!ptx::mbar_wait_s<true>(&tile_full[slot], use & 1, st)) break;
          t = tile_ring[slot];
        }
        if (t >= ntiles) break;
        int sidx, row, c;
        TcStudy S;
        decode_tile(b, t, sidx, row, c, S);
        const TcMaps& M = b.maps[sidx];
        const pair2::Unit u = pair2::make_unit(row, S);
        const int ycol = c * TN + (int)rank * (TN / 2);  // this CTA's SNP columns
        if (!ptx::mbar_wait(x8_empty, (x8n & 1) ^ 1, st)) break;
        ptx::mbar_arrive_expect_tx(x8_full, (u.paired ? 2 : 1) * K::X8H_BYTES);
        ptx::tma_load_2d(x8, &M.X8H, x8_full, u.k0 * TB, ycol);
        if (u.paired) ptx::tma_load_2d(x8 + K::X8H_BYTES, &M.X8H, x8_full, (u.k0 + 1) * TB, ycol);
        ++x8n;
        bool ok = true;
        for (int jj = 0; jj < u.nkb && ok; ++jj) {
          int j, arow;
          const pair2::Kind kind = pair2::kind_of(u, rank, jj, j, arow);
          const bool btma = kind == pair2::MJ;  // else B is cast from int8
          if (btma) {
            if (!ptx::wait_flag(&S.flags[j * S.C + c], st)) { ok = false; break; }
            ptx::fence_proxy_async_global();
          }
          const int ay = arow >= 0 ? arow * TB : -TB;  // -TB: wholly outside, reads zeros
          for (int h = 0; h < K::CPB; ++h, ++cnt) {
            const int s = cnt % ST;
            const uint32_t r = cnt / ST;
            if (!ptx::mbar_wait(&empty[s], (r & 1) ^ 1, st)) { ok = false; break; }
            uint8_t* sb = smem + s * K::STAGE_BYTES;
            const int kx = j * TB + h * K::KCH;
            const uint32_t fb = lead_addr(&full[s]);
            if (leader)
              ptx::mbar_arrive_expect_tx(&full[s], 2 * (2 * K::A_BYTES + (btma ? 2 * K::B_BYTES : 0)));
            else
              ptx::mbar_arrive_peer_count(fb);
            ptx::tma_load_2d_pair(sb, &M.Ahi, fb, kx, ay);
            ptx::tma_load_2d_pair(sb + K::A_BYTES, &M.Alo, fb, kx, ay);
            if (btma) {
              ptx::tma_load_2d_pair(sb + 2 * K::A_BYTES, &M.BhiH, fb, kx, ycol);
              ptx::tma_load_2d_pair(sb + 2 * K::A_BYTES + K::B_BYTES, &M.BloH, fb, kx, ycol);
              count_lead(&full[s]);
            }
          }
        }
        if (!ok) break;
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------- MMA issuer (CTA 0 only)
    if (lane == 0) {
      constexpr uint32_t idesc = ptx::idesc_f32acc<TF32>(2 * TB, TN);
      uint32_t cnt = 0, kb = 0;
      for (int it = 0;; ++it) {
        const int slot = it % TRING;
        const uint32_t use = it / TRING;
        if (!ptx::mbar_wait_s<true>(&tile_full[slot], use & 1, st)) break;
        const int t = tile_ring[slot];
        ptx::mbar_arrive(&tile_empty[slot]);
        if (t >= ntiles) break;
        if (!leader) continue;
        int sidx, row, c;
        TcStudy S;
        decode_tile(b, t, sidx, row, c, S);
        const pair2::Unit u = pair2::make_unit(row, S);
        bool ok = true;
        int q = 0, a = 0;
        uint32_t d = 0, accumulate = 0;
        for (int jj = 0; jj < u.nkb && ok; ++jj) {
          int j, arow;
          const pair2::Kind kind = pair2::kind_of(u, rank, jj, j, arow);
          if (q % PROMOTE == 0) {
            // a fresh partial every PROMOTE K-blocks
            a = kb & 1;
            if (!ptx::mbar_wait(&part_empty[a], ((kb >> 1) & 1) ^ 1, st)) { ok = false; break; }
            ++kb;
            ptx::tc_fence_after();
            d = tmem_base + a * TN;
            accumulate = 0;
          }
          const bool three = kind == pair2::MJ;  // X~ has a lo piece
          for (int h = 0; h < K::CPB; ++h, ++cnt) {
            const int s = cnt % ST;
            const uint32_t r = cnt / ST;
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
              ptx::mma_pair<TF32>(d, alo, bhi, idesc, accumulate);
              accumulate = 1;
              if (three) ptx::mma_pair<TF32>(d, ahi, blo, idesc, 1);
              ptx::mma_pair<TF32>(d, ahi, bhi, idesc, 1);
            }
            ptx::mma_commit_pair(&empty[s], BOTH);
          }
          if (!ok) break;
          if (q % PROMOTE == PROMOTE - 1 || jj == u.nkb - 1) ptx::mma_commit_pair(&part_full[a], BOTH);
          ++q;
        }
        if (!ok) break;
      }
    }
  } else if (warp < 4) {
    // ----------------------- int8 -> BF16/TF32 cast of D0 and D1 (this CTA's columns)
    const int ct = threadIdx.x - 64;  // 0..63
    constexpr int E = 16 / K::ESZ;    // elements per 16-byte chunk
    uint32_t cnt = 0, x8n = 0;
    for (int it = 0;; ++it) {
      const int slot = it % TRING;
      const uint32_t use = it / TRING;
      if (!ptx::group_and(2, 64, ptx::mbar_wait_s<true>(&tile_full[slot], use & 1, st))) break;
      const int t = tile_ring[slot];
      ptx::named_bar(2, 64);
      if (lane == 0) ptx::mbar_arrive(&tile_empty[slot]);
      if (t >= ntiles) break;
      int sidx, row, ctile;
      TcStudy S;
      decode_tile(b, t, sidx, row, ctile, S);
      const pair2::Unit u = pair2::make_unit(row, S);
      if (!ptx::group_and(2, 64, ptx::mbar_wait(x8_full, x8n & 1, st))) break;
      bool ok = true;
      const int nd = u.paired ? 2 : 1;  // D0, D1
      for (int dd = 0; dd < nd && ok; ++dd) {
        const int panel = u.k0 + dd;
        for (int h = 0; h < K::CPB; ++h) {
          const uint32_t pos = cnt + dd * K::CPB + h;
          const int s = pos % ST;
          const uint32_t r = pos / ST;
          if (!ptx::group_and(2, 64, ptx::mbar_wait(&empty[s], (r & 1) ^ 1, st))) { ok = false; break; }
          uint8_t* bh = smem + s * K::STAGE_BYTES + 2 * K::A_BYTES;
          for (int col = ct; col < TN / 2; col += 64) {
            const int8_t* src = reinterpret_cast<const int8_t*>(x8 + dd * K::X8H_BYTES + col * TB + h * K::KCH);
            const int colg = ctile * TN + (int)rank * (TN / 2) + col;
            const int csh = (S.shift && colg < S.ncols) ? S.shift[colg] : 0;
            const int row0 = panel * TB + h * K::KCH;
#pragma unroll
            for (int q = 0; q < 4; ++q) {  // four 16-byte chunks per 64-byte row
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
              *reinterpret_cast<uint4*>(bh + col * 64 + ((q ^ ((col >> 1) & 3)) << 4)) =
                  make_uint4(w[0], w[1], w[2], w[3]);
            }
          }
          ptx::fence_proxy_async_shared();
          ptx::named_bar(2, 64);
          // the pair's tensor cores read these generic writes: cluster-scope release
          if (ct == 0) {
            if (leader)
              ptx::mbar_arrive(&full[s]);
            else
              ptx::mbar_arrive_peer(ptx::peer_addr(&full[s], 0));
          }
        }
      }
      if (!ok) break;
      if (ct == 0) ptx::mbar_arrive(x8_empty);
      ++x8n;
      cnt += K::CPB * u.nkb;
    }
  } else {
    // ----------------------------------------------------------------- epilogue
    constexpr int NT = 32 * EPI_WARPS;
    const int e = warp - 4;
    const int lq = e & 3;
    const int chalf = e >> 2;
    uint32_t kb = 0, gq = 0;  // partials taken; store chunks issued
    float master[EPI_COLS];
    for (int it = 0;; ++it) {
      const int slot = it % TRING;
      const uint32_t use = it / TRING;
      if (!ptx::group_and(1, NT, ptx::mbar_wait_s<true>(&tile_full[slot], use & 1, st))) break;
      const int t = tile_ring[slot];
      ptx::named_bar(1, NT);
      if (lane == 0) ptx::mbar_arrive(&tile_empty[slot]);
      if (t >= ntiles) break;
      int sidx, row, c;
      TcStudy S;
      decode_tile(b, t, sidx, row, c, S);
      const pair2::Unit u = pair2::make_unit(row, S);
      const bool has = leader || u.paired;  // this CTA has a tile
      const int k = u.k0 + (int)rank;
      const int npm = (u.nkb + PROMOTE - 1) / PROMOTE;  // shared partials
#pragma unroll
      for (int i = 0; i < EPI_COLS; ++i) master[i] = 0.f;
      // waits for partial kb, adds it into the master when `add`, hands it back to CTA 0
      auto take = [&](bool add) -> bool {
        const int a = kb & 1;
        if (!ptx::group_and(1, NT, ptx::mbar_wait(&part_full[a], (kb >> 1) & 1, st))) return false;
        ptx::tc_fence_after();
        if (add) {
          const uint32_t tb = tmem_base + (static_cast<uint32_t>(32 * lq) << 16) + a * TN + chalf * EPI_COLS;
#pragma unroll
          for (int ch = 0; ch < EPI_COLS / 16; ++ch) {
            uint32_t v[16];
            ptx::tmem_ld_32x32b_x16(tb + ch * 16, v);
            ptx::tmem_ld_wait();
#pragma unroll
            for (int i = 0; i < 16; ++i) master[ch * 16 + i] += __uint_as_float(v[i]);  // round to nearest
          }
        }
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) count_lead(&part_empty[a]);
        ++kb;
        return true;
      };
      // X~ of this CTA's tile to HBM by TMA stores of shared-memory chunks.
      // The MMA operand pieces go first (BF16: hi, lo; TF32: the FP32 value,
      // read as TF32 hi, and lo), then the tile's finished-flag; in BF16 mode
      // the FP32 copy for the reductions follows off the dependency chain.
      auto publish = [&]() {
        constexpr int CC = pair2::st_cols<TF32>();
        const TcMaps& M = b.maps[sidx];
        uint8_t* stg = smem + K::STG_OFF + e * 2 * K::CHUNK_BYTES;
        const int r0 = k * TB + 32 * lq;
        const int c0 = c * TN + chalf * EPI_COLS;
        // the next staging buffer, once the store group that last read it is done
        auto next_buf = [&]() -> uint8_t* {
          uint8_t* buf = stg + (gq & 1) * K::CHUNK_BYTES;
          if (gq >= 2) {
            if (lane == 0) ptx::bulk_wait_read<1>();
            __syncwarp();
          }
          ++gq;
          return buf;
        };
#pragma unroll
        for (int q = 0; q < EPI_COLS / CC; ++q) {
          uint8_t* buf = next_buf();
#pragma unroll
          for (int i = 0; i < CC; ++i) {
            const float x = master[q * CC + i];
            if constexpr (TF32) {
              reinterpret_cast<float*>(buf)[i * 32 + lane] = x;
              reinterpret_cast<float*>(buf + 1024)[i * 32 + lane] = x - __uint_as_float(tf32_trunc_bits(x));
            } else {
              const __nv_bfloat16 hi = __float2bfloat16_rn(x);
              reinterpret_cast<__nv_bfloat16*>(buf)[i * 32 + lane] = hi;
              reinterpret_cast<__nv_bfloat16*>(buf + 1024)[i * 32 + lane] =
                  __float2bfloat16_rn(x - __bfloat162float(hi));
            }
          }
          ptx::fence_proxy_async_shared();
          __syncwarp();
          if (lane == 0) {
            const int y = c0 + q * CC;
            ptx::tma_store_2d(TF32 ? &M.StX : &M.StHi, buf, r0, y);
            ptx::tma_store_2d(&M.StLo, buf + 1024, r0, y);
            ptx::bulk_commit();
          }
        }
        if (lane == 0) {
          // this warp's operand stores are complete and visible device-wide before the flag
          ptx::bulk_wait_all();
          ptx::fence_proxy_async_global();
          asm volatile("fence.acq_rel.gpu;" ::: "memory");
        }
        __syncwarp();
        ptx::named_bar(1, NT);
        if (e == 0 && lane == 0) ptx::st_release(&S.flags[k * S.C + c], 1);
        if constexpr (!TF32) {
#pragma unroll
          for (int q = 0; q < EPI_COLS / CC; ++q) {
            uint8_t* buf = next_buf();
#pragma unroll
            for (int i = 0; i < CC; ++i) reinterpret_cast<float*>(buf)[i * 32 + lane] = master[q * CC + i];
            ptx::fence_proxy_async_shared();
            __syncwarp();
            if (lane == 0) {
              ptx::tma_store_2d(&M.StX, buf, r0, c0 + q * CC);
              ptx::bulk_commit();
            }
          }
        }
      };
      bool ok = true;
      for (int pp = 0; pp < npm && ok; ++pp) ok = take(has);
      if (!ok) break;
      if (has) publish();
    }
    if (lane == 0) ptx::bulk_wait_all();  // the last stores have read the staging buffers
  }

  // ---------------------------------------------------------------- teardown
  if (warp == 1 && lane == 0 && leader) {
    // every MMA of the pair has completed before tensor memory is released
    ptx::mma_commit_pair(drain, 1);
    const long long t0 = ptx::globaltimer();
    while (!ptx::mbar_try_wait(drain, 0) && ptx::globaltimer() - t0 < 100000000LL) {
    }
  }
  if (ptx::aborting(st)) {
    const long long t0 = ptx::globaltimer();
    while (ptx::globaltimer() - t0 < 2000000LL) {
    }
  }
  // neither CTA retires (or frees tensor memory) while the other may still
  // read its shared memory, arrive on its barriers or write its partials
  ptx::cluster_sync();
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  if (warp == 2) ptx::tmem_dealloc_pair(tmem_base, 2 * TN);
}

// ------------------------------------------------------------- inverse form
// Tile mode TILES_INVERSE: the substitution moved into set-up.  L^-1 (lower
// triangular, n_pad x n_pad, row-major) is formed once per study and split
// into hi + lo pieces; a block of SNP columns is then the triangular product
//     X~_kc = sum_{j<=k} (L^-1)_kj X_jc
// whose output tiles depend on nothing but the inputs.  The dosages are exact
// in BF16/TF32, so each K-block takes the two products Linv_hi X + Linv_lo X.
// Work units are the row-panel pairs (2u, 2u+1) of a strip as one M = 256
// product on a 2-SM cluster (cta_group::2, as in the pair product), handed out
// longest first.  B comes by TMA from the cast copy of the block
// (cast_shift_kernel: x - c_i as BF16/FP32), so TMA alone fills every stage.
namespace inv2 {
// Fused sums: the staging of one epilogue warp (4 KB) holds a transposition
// buffer for 32 rows x 16 columns and, from FS_W_OFF, the warp's 32 rows of W.
// Rows 0..15 sit at row * 20 floats, rows 16..31 at 336 + (row - 16) * 20:
// a row's 16 floats go in as four 16-byte stores (8 lanes per phase on 32
// distinct banks) and a column comes out with lanes 0..15 on rows 0..15 and
// lanes 16..31 on rows 16..31 (banks c and 16 + c).
constexpr int FS_W_OFF = 2688;
__device__ __forceinline__ int fs_idx(int row, int col) { return (row & 15) * 20 + (row >> 4) * 336 + col; }
static_assert((336 + 15 * 20 + 16) * 4 <= FS_W_OFF && FS_W_OFF + 32 * 8 * 4 <= 4096, "fused-sum staging");

// The per-SNP sums of Listing 1 over one CTA's 128 rows of a tile, formed in
// place of storing X~: per SNP column, x~ . W[:, a] (a < nw) and x~ . x~.
// master holds this lane's row (the epilogue warp's 32 rows x 128 columns)
// before its scale rs (the FP16 form's power of two; else 1).  16 columns at
// a time go through the warp's transposition buffer; lane (ci, h) sums rows
// 16h .. 16h+15 of column ci in FP32 FMAs (packed in pairs) and one shuffle
// adds the halves.
// WS = 4 (nw <= 4): the four row quarters (warps lq = 0..3 of the same column
// half) then add their 32-row sums through shared memory in a fixed order and
// write one plane per (row panel k, quantity a): red[(k (nw+1) + a) ldr + j].
// WS = 8: each warp writes its 32-row sums, plane ((4k + lq)(nw+1) + a).
// `grp` is the staging of warp lq = 0 of this column half (warp lq's at
// grp + 4 KB lq); named barrier 2 + chalf holds the half's 4 warps.
template <int WS>
__device__ __forceinline__ void tile_sums(const float (&master)[EPI_COLS], float rs, uint8_t* grp, int lq, int chalf,
                                          float* red, int64_t ldr, int k, int nw, int lane, int cols_left) {
  const int ci = lane & 15, h = lane >> 4;
  uint8_t* stg = grp + lq * 2 * 2048;
  float* sm = reinterpret_cast<float*>(stg);
  const float* wsm = reinterpret_cast<const float*>(stg + FS_W_OFF);
  const int nq = nw + 1;
  float keep[4][WS + 1];  // WS = 4: this lane's half of the chunks' sums (chunks 4h .. 4h+3)
#pragma unroll
  for (int q = 0; q < EPI_COLS / 16; ++q) {
    float4* dst = reinterpret_cast<float4*>(sm + fs_idx(lane, 0));
#pragma unroll
    for (int j = 0; j < 4; ++j)
      dst[j] = make_float4(master[q * 16 + 4 * j] * rs, master[q * 16 + 4 * j + 1] * rs,
                           master[q * 16 + 4 * j + 2] * rs, master[q * 16 + 4 * j + 3] * rs);
    __syncwarp();
    float acc[WS + 1];
#pragma unroll
    for (int a = 0; a <= WS; ++a) acc[a] = 0.f;
#pragma unroll 2
    for (int r = 0; r < 16; ++r) {
      const float x = sm[fs_idx(16 * h + r, ci)];
      const float4* wr = reinterpret_cast<const float4*>(wsm + (16 * h + r) * WS);
#pragma unroll
      for (int v = 0; v < WS / 4; ++v) {
        const float4 w = wr[v];
        ptx::fma2(acc[4 * v], acc[4 * v + 1], x, w.x, w.y);
        ptx::fma2(acc[4 * v + 2], acc[4 * v + 3], x, w.z, w.w);
      }
      acc[WS] = fmaf(x, x, acc[WS]);
    }
#pragma unroll
    for (int a = 0; a <= WS; ++a) acc[a] += __shfl_xor_sync(0xffffffffu, acc[a], 16);
    if constexpr (WS == 4) {
#pragma unroll
      for (int a = 0; a <= WS; ++a) keep[q & 3][a] = (h == (q >> 2)) ? acc[a] : keep[q & 3][a];
    } else {
      float* out = red + (int64_t)(4 * k + lq) * nq * ldr + q * 16 + ci;
      if (h == 0 && q * 16 + ci < cols_left) {
#pragma unroll
        for (int a = 0; a < WS; ++a)
          if (a < nw) out[a * ldr] = acc[a];
        out[nw * ldr] = acc[WS];
      }
    }
    __syncwarp();
  }
  if constexpr (WS == 4) {
    // exchange: this warp's sums at [chunk][a][column] in its transposition
    // buffer (8 x 5 x 16 floats), then warp lq adds chunks 2lq, 2lq+1 over the
    // four row quarters in order 0..3 and writes the panel's plane
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int a = 0; a <= WS; ++a) sm[((4 * h + j) * (WS + 1) + a) * 16 + ci] = keep[j][a];
    auto half_bar = [&] {  // the 4 warps of this column half
      if (chalf == 0)
        ptx::named_bar(2, 128);
      else
        ptx::named_bar(3, 128);
    };
    half_bar();
    const int q = 2 * lq + h;
    if (q * 16 + ci < cols_left) {
      float* out = red + (int64_t)k * nq * ldr + q * 16 + ci;
#pragma unroll
      for (int a = 0; a <= WS; ++a) {
        float v = 0.f;
#pragma unroll
        for (int w = 0; w < 4; ++w) v += reinterpret_cast<const float*>(grp + w * 2 * 2048)[(q * (WS + 1) + a) * 16 + ci];
        if (a < nw) out[a * ldr] = v;
        if (a == WS) out[nw * ldr] = v;
      }
    }
    half_bar();  // the buffers are free for the next tile
  }
}

// NST 64-byte K-steps of operands in flight (8, the most that fit beside the
// epilogue staging, or 6: a batch's autotuner picks one), two to a stage: the
// single MMA-issuing thread waits on a stage and commits it once per eight
// MMAs (one step a stage, four MMAs, ran 4 % slower in BF16/FP16, 10 % in TF32)
template <bool TF32, int NST = 8>
struct Cfg {
  static constexpr int SUB = 2;  // K-steps per stage
  static constexpr int STAGES = NST / SUB;
  static constexpr int ESZ = TF32 ? 4 : 2;
  static constexpr int KCH = 64 / ESZ;  // K per step
  static constexpr int KMMA = TF32 ? 8 : 16;
  static constexpr int CPB = TB / (KCH * SUB);  // stages per TB-wide K-block
  static constexpr int A_BYTES = TB * 64;                    // one piece of this CTA's L^-1 rows: 8 KB
  static constexpr int B_BYTES = (TN / 2) * 64;              // this CTA's half of the SNP columns: 8 KB
  static constexpr int STEP_BYTES = 2 * A_BYTES + B_BYTES;   // 24 KB: [hi | lo | x]
  static constexpr int STAGE_BYTES = SUB * STEP_BYTES;       // 48 KB
  static constexpr int CHUNK_BYTES = 2048;
  static constexpr int STG_OFF = STAGES * STAGE_BYTES;
  static constexpr int BAR_OFF = STG_OFF + EPI_WARPS * 2 * CHUNK_BYTES;
  static constexpr int NBARS = 2 * STAGES + 4 + 3 * TRING + 1;
  static constexpr int SMEM = 1024 + BAR_OFF + NBARS * 8 + TRING * 4 + 16;
  static_assert(SMEM <= 232448, "shared memory per CTA");
  static_assert(CHUNK_BYTES == 2048, "the fused sums take 4 KB of staging per epilogue warp");
};
}  // namespace inv2

// F16 (with TF32 false): L^-1 pieces and the cast block are FP16; row r of
// L^-1 was scaled by 1 / rscale[r] (a power of two) before the split, so the
// epilogue multiplies its results back by rscale[r].
template <bool TF32, bool F16 = false, int NST = 8>
__global__ void __launch_bounds__(THREADS, 1) trsm_tc_inv_kernel(const __grid_constant__ TcBatch b) {
  using K = inv2::Cfg<TF32, NST>;
  constexpr int ST = K::STAGES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + K::BAR_OFF);
  uint64_t* full = bars;                 // CTA 0: both CTAs' loads of a stage
  uint64_t* empty = full + ST;           // CTA 0's commit: the stage's MMAs are done
  uint64_t* part_full = empty + ST;      // CTA 0's commit: a partial is complete
  uint64_t* part_empty = part_full + 2;  // CTA 0: both CTAs' epilogues are done with a partial
  uint64_t* tile_full = part_empty + 2;
  uint64_t* tile_empty = tile_full + TRING;
  uint64_t* peer_free = tile_empty + TRING;
  uint64_t* drain = peer_free + TRING;
  int* tile_ring = reinterpret_cast<int*>(drain + 1);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tile_ring + TRING);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = b.ntiles;  // work units: row-panel pairs of a strip
  DevStatus* st = b.st;
  const uint32_t rank = ptx::cluster_ctarank();
  const bool leader = rank == 0;
  constexpr uint16_t BOTH = 3;
  auto lead_addr = [&](uint64_t* bar) -> uint32_t { return leader ? ptx::smem_u32(bar) : ptx::peer_addr(bar, 0); };
  auto count_lead = [&](uint64_t* bar) {
    if (leader)
      ptx::mbar_arrive(bar);
    else
      ptx::mbar_arrive_peer_count(ptx::peer_addr(bar, 0));
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) {
      ptx::mbar_init(&full[s], 2);   // one arrival from each CTA's producer (+ the bytes of both)
      ptx::mbar_init(&empty[s], 1);  // CTA 0's commit
    }
    for (int a = 0; a < 2; ++a) {
      ptx::mbar_init(&part_full[a], 1);
      ptx::mbar_init(&part_empty[a], 2 * EPI_WARPS);
    }
    for (int i = 0; i < TRING; ++i) {
      ptx::mbar_init(&tile_full[i], 1);
      ptx::mbar_init(&tile_empty[i], 1 + EPI_WARPS);
      ptx::mbar_init(&peer_free[i], 1);
    }
    ptx::mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int q = 0; q < b.nstudies; ++q) {
      ptx::prefetch_tensormap(&b.maps[q].Ahi);
      ptx::prefetch_tensormap(&b.maps[q].Alo);
      ptx::prefetch_tensormap(&b.maps[q].XcH);
    }
  }
  if (warp == 2) {
    ptx::tmem_alloc_pair(tmem_slot, 2 * TN);
    ptx::tmem_relinquish_pair();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  ptx::cluster_sync();  // both CTAs' barriers and tensor memory exist before any remote access
  const uint32_t tmem_base = *tmem_slot;
  // launched as a dependent of the cast pre-pass: set-up above overlaps its
  // tail; no global memory is touched before it has completed
  ptx::griddep_wait();

  if (warp == 0) {
    // ------------------------------------------------ scheduler + TMA producer
    if (lane == 0) {
      uint32_t cnt = 0;
      for (int it = 0;; ++it) {
        const int slot = it % TRING;
        const uint32_t use = it / TRING;
        if (!ptx::mbar_wait(&tile_empty[slot], (use & 1) ^ 1, st)) break;
        int t;
        if (leader) {
          if (!ptx::mbar_wait(&peer_free[slot], use & 1, st)) break;
          t = ptx::aborting(st) ? ntiles : (int)atomicAdd(b.counter, 1u);
          if (t > ntiles) t = ntiles;
          tile_ring[slot] = t;
          ptx::st_peer_u32(ptx::peer_addr(&tile_ring[slot], 1), (uint32_t)t);
          ptx::mbar_arrive(&tile_full[slot]);
          ptx::mbar_arrive_peer(ptx::peer_addr(&tile_full[slot], 1));
        } else {
          ptx::mbar_arrive_peer(ptx::peer_addr(&peer_free[slot], 0));
          if (!ptx::mbar_wait_s<true>(&tile_full[slot], use & 1, st)) break;
          t = tile_ring[slot];
        }
        if (t >= ntiles) {
          ptx::griddep_launch();  // no more units for this CTA: the sums' kernel may launch
          break;
        }
        int sidx, row, c;
        TcStudy S;
        decode_tile(b, t, sidx, row, c, S);
        const TcMaps& M = b.maps[sidx];
        const pair2::Unit u = pair2::make_unit_inv(row, S);
        const int arow = rank == 0 ? u.k0 : (u.paired ? u.k0 + 1 : -1);  // this CTA's row panel
        const int ycol = c * TN + (int)rank * (TN / 2);                   // this CTA's SNP columns
        bool ok = true;
        for (int j = 0; j < u.nkb && ok; ++j) {  // the unit's K-blocks
          // a block above the diagonal, or no rows: a box wholly outside reads zeros
          const int ay = (arow >= 0 && j <= arow) ? arow * TB : -TB;
          for (int h = 0; h < K::CPB; ++h, ++cnt) {
            const int s = cnt % ST;
            const uint32_t r = cnt / ST;
            if (!ptx::mbar_wait(&empty[s], (r & 1) ^ 1, st)) { ok = false; break; }
            uint8_t* sb = smem + s * K::STAGE_BYTES;
            const int kx = j * TB + h * K::KCH * K::SUB;
            const uint32_t fb = lead_addr(&full[s]);
            if (leader)
              ptx::mbar_arrive_expect_tx(&full[s], 2 * K::STAGE_BYTES);
            else
              ptx::mbar_arrive_peer_count(fb);
#pragma unroll
            for (int u2 = 0; u2 < K::SUB; ++u2) {
              uint8_t* sp = sb + u2 * K::STEP_BYTES;
              ptx::tma_load_2d_pair(sp, &M.Ahi, fb, kx + u2 * K::KCH, ay);
              ptx::tma_load_2d_pair(sp + K::A_BYTES, &M.Alo, fb, kx + u2 * K::KCH, ay);
              ptx::tma_load_2d_pair(sp + 2 * K::A_BYTES, &M.XcH, fb, kx + u2 * K::KCH, ycol);
            }
          }
        }
        if (!ok) break;
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------- MMA issuer (CTA 0 only)
    if (lane == 0) {
      constexpr uint32_t idesc = F16 ? ptx::idesc_f32acc_f16(2 * TB, TN) : ptx::idesc_f32acc<TF32>(2 * TB, TN);
      uint32_t cnt = 0, kb = 0;
      for (int it = 0;; ++it) {
        const int slot = it % TRING;
        const uint32_t use = it / TRING;
        if (!ptx::mbar_wait_s<true>(&tile_full[slot], use & 1, st)) break;
        const int t = tile_ring[slot];
        ptx::mbar_arrive(&tile_empty[slot]);
        if (t >= ntiles) break;
        if (!leader) continue;
        int sidx, row, c;
        TcStudy S;
        decode_tile(b, t, sidx, row, c, S);
        const pair2::Unit u = pair2::make_unit_inv(row, S);
        const int nkb = u.nkb;
        bool ok = true;
        int a = 0;
        uint32_t d = 0, accumulate = 0;
        for (int j = 0; j < nkb && ok; ++j) {
          // K-blocks 0 and 1 of a unit into one partial, every later K-block
          // into a fresh one (promoted by the epilogue): three K-blocks of work
          // before the epilogue must take a partial, to cover its tile-end sums
          if (j != 1) {
            a = kb & 1;
            if (!ptx::mbar_wait(&part_empty[a], ((kb >> 1) & 1) ^ 1, st)) { ok = false; break; }
            ++kb;
            ptx::tc_fence_after();
            d = tmem_base + a * TN;
            accumulate = 0;
          }
          for (int h = 0; h < K::CPB; ++h, ++cnt) {
            const int s = cnt % ST;
            const uint32_t r = cnt / ST;
            if (!ptx::mbar_wait(&full[s], r & 1, st)) { ok = false; break; }
            ptx::tc_fence_after();
            const uint32_t base0 = ptx::smem_u32(smem + s * K::STAGE_BYTES);
#pragma unroll
            for (int u2 = 0; u2 < K::SUB; ++u2) {
              const uint32_t base = base0 + u2 * K::STEP_BYTES;
#pragma unroll
              for (int kk = 0; kk < K::KCH / K::KMMA; ++kk) {
                const uint32_t off = kk * K::KMMA * K::ESZ;
                const uint64_t ahi = ptx::sdesc_k64(base + off);
                const uint64_t alo = ptx::sdesc_k64(base + K::A_BYTES + off);
                const uint64_t bx = ptx::sdesc_k64(base + 2 * K::A_BYTES + off);
                ptx::mma_pair<TF32>(d, alo, bx, idesc, accumulate);
                accumulate = 1;
                ptx::mma_pair<TF32>(d, ahi, bx, idesc, 1);
              }
            }
            ptx::mma_commit_pair(&empty[s], BOTH);
          }
          if (!ok) break;
          if (j != 0 || nkb == 1) ptx::mma_commit_pair(&part_full[a], BOTH);
        }
        if (!ok) break;
      }
    }
  } else if (warp >= 4) {
    // ----------------------------------------------------------------- epilogue
    constexpr int NT = 32 * EPI_WARPS;
    constexpr int CC = inv2::ST_COLS;
    const int e = warp - 4;
    const int lq = e & 3;
    const int chalf = e >> 2;
    uint32_t kb = 0, gq = 0;  // partials taken; store chunks issued
    float master[EPI_COLS];
    for (int it = 0;; ++it) {
      const int slot = it % TRING;
      const uint32_t use = it / TRING;
      if (!ptx::group_and(1, NT, ptx::mbar_wait_s<true>(&tile_full[slot], use & 1, st))) break;
      const int t = tile_ring[slot];
      ptx::named_bar(1, NT);
      if (lane == 0) ptx::mbar_arrive(&tile_empty[slot]);
      if (t >= ntiles) break;
      int sidx, row, c;
      TcStudy S;
      decode_tile(b, t, sidx, row, c, S);
      const pair2::Unit u = pair2::make_unit_inv(row, S);
      const bool has = leader || u.paired;  // this CTA has a tile
      const int k = u.k0 + (int)rank;
      uint8_t* stg = smem + K::STG_OFF + e * 2 * K::CHUNK_BYTES;  // this warp's 4 KB of staging
      if (S.red && has) {
        // fused sums: this warp's 32 rows of W into its staging (read at the
        // tile's end; the copies land while the partials are added)
        if (gq > 0) {  // stores of an earlier tile still reading the staging buffers
          if (lane == 0) ptx::bulk_wait_read<0>();
          __syncwarp();
        }
        const float* wsrc = S.w32 + (int64_t)(k * TB + 32 * lq + lane) * S.ws;
        float* wdst = reinterpret_cast<float*>(stg + inv2::FS_W_OFF) + lane * S.ws;
        for (int v = 0; v < S.ws; v += 4) ptx::cp_async16(wdst + v, wsrc + v);
        ptx::cp_async_commit();
      }
#pragma unroll
      for (int i = 0; i < EPI_COLS; ++i) master[i] = 0.f;
      bool ok = true;
      const int nkb = u.nkb;
      const int nparts = nkb > 1 ? nkb - 1 : 1;  // K-blocks 0 and 1 share a partial
      for (int pp = 0; pp < nparts && ok; ++pp) {
        const int a = kb & 1;
        if (!ptx::group_and(1, NT, ptx::mbar_wait(&part_full[a], (kb >> 1) & 1, st))) { ok = false; break; }
        ptx::tc_fence_after();
        if (has) {
          const uint32_t tb = tmem_base + (static_cast<uint32_t>(32 * lq) << 16) + a * TN + chalf * EPI_COLS;
#pragma unroll
          for (int ch = 0; ch < EPI_COLS / 16; ++ch) {
            uint32_t v[16];
            ptx::tmem_ld_32x32b_x16(tb + ch * 16, v);
            ptx::tmem_ld_wait();
#pragma unroll
            for (int i = 0; i < 16; ++i) master[ch * 16 + i] += __uint_as_float(v[i]);  // round to nearest
          }
        }
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) count_lead(&part_empty[a]);
        ++kb;
      }
      if (!ok) break;
      if (!has) continue;
      // X~ of this CTA's tile to HBM by TMA stores of shared-memory chunks
      const TcMaps& M = b.maps[sidx];
      const int r0 = k * TB + 32 * lq;
      const int c0 = c * TN + chalf * EPI_COLS;
      // F16: this thread's row back to the scale of L^-1 (exact: a power of two)
      const float rs = F16 ? __ldg(S.rscale + r0 + lane) : 1.f;
      if (S.red) {
        // the per-SNP sums of Listing 1 in place of the store
        ptx::cp_async_wait_all();  // this lane's W row
        __syncwarp();
        uint8_t* grp = smem + K::STG_OFF + 4 * chalf * 2 * K::CHUNK_BYTES;
        if (S.ws == 4)
          inv2::tile_sums<4>(master, rs, grp, lq, chalf, S.red + c0, S.ldr, k, S.nw, lane, S.ncols - c0);
        else
          inv2::tile_sums<8>(master, rs, grp, lq, chalf, S.red + c0, S.ldr, k, S.nw, lane, S.ncols - c0);
        continue;
      }
      if constexpr (F16) {
#pragma unroll
        for (int i = 0; i < EPI_COLS; ++i) master[i] *= rs;
      }
      auto next_buf = [&]() -> uint8_t* {
        uint8_t* buf = stg + (gq & 1) * K::CHUNK_BYTES;
        if (gq >= 2) {
          if (lane == 0) ptx::bulk_wait_read<1>();
          __syncwarp();
        }
        ++gq;
        return buf;
      };
#pragma unroll
      for (int q = 0; q < EPI_COLS / CC; ++q) {
        uint8_t* buf = next_buf();
#pragma unroll
        for (int i = 0; i < CC; ++i) reinterpret_cast<float*>(buf)[i * 32 + lane] = master[q * CC + i];
        ptx::fence_proxy_async_shared();
        __syncwarp();
        if (lane == 0) {
          ptx::tma_store_2d(&M.StX, buf, r0, c0 + q * CC);
          ptx::bulk_commit();
        }
      }
    }
    if (lane == 0) ptx::bulk_wait_all();  // the last stores have read the staging buffers
  }

  // ---------------------------------------------------------------- teardown
  if (warp == 1 && lane == 0 && leader) {
    // every MMA of the pair has completed before tensor memory is released
    ptx::mma_commit_pair(drain, 1);
    const long long t0 = ptx::globaltimer();
    while (!ptx::mbar_try_wait(drain, 0) && ptx::globaltimer() - t0 < 100000000LL) {
    }
  }
  if (ptx::aborting(st)) {
    const long long t0 = ptx::globaltimer();
    while (ptx::globaltimer() - t0 < 2000000LL) {
    }
  }
  ptx::cluster_sync();
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  if (warp == 2) ptx::tmem_dealloc_pair(tmem_base, 2 * TN);
}

// ------------------------------------------------------------ launch entries
template <bool TF32>
static cudaLaunchConfig_t pair_config(cudaLaunchAttribute* attr, int grid, cudaStream_t s, TileMode mode,
                                      int stages = 8) {
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof cfg);
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(THREADS);
  cfg.dynamicSmemBytes = mode != TILES_INVERSE ? pair2::Cfg<TF32>::SMEM
                         : stages == 6         ? inv2::Cfg<TF32, 6>::SMEM
                                               : inv2::Cfg<TF32>::SMEM;
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

template <bool TF32>
static cudaError_t set_attrs(bool clusters) {
  constexpr cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(trsm_tc_kernel<TF32>, A, Cfg<TF32>::SMEM);
  if (e != cudaSuccess || !clusters) return e;
  if ((e = cudaFuncSetAttribute(trsm_tc_pair_mma_kernel<TF32>, A, pair2::Cfg<TF32>::SMEM)) != cudaSuccess) return e;
  if (!TF32 && (e = cudaFuncSetAttribute(trsm_tc_inv_kernel<false, true>, A, inv2::Cfg<false>::SMEM)) != cudaSuccess)
    return e;
  if (!TF32 &&
      (e = cudaFuncSetAttribute(trsm_tc_inv_kernel<false, true, 6>, A, inv2::Cfg<false, 6>::SMEM)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(trsm_tc_inv_kernel<TF32, false, 6>, A, inv2::Cfg<TF32, 6>::SMEM)) != cudaSuccess)
    return e;
  return cudaFuncSetAttribute(trsm_tc_inv_kernel<TF32>, A, inv2::Cfg<TF32>::SMEM);
}

cudaError_t set_kernel_attrs(bool tf32, bool clusters) {
  return tf32 ? set_attrs<true>(clusters) : set_attrs<false>(clusters);
}

template <bool TF32>
static cudaError_t clusters_of(int num_sms, TileMode mode, int* out, bool f16) {
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = pair_config<TF32>(attr, 2 * (num_sms / 2), nullptr, mode);
  const void* fn = mode == TILES_INVERSE ? (f16 ? (const void*)trsm_tc_inv_kernel<false, true>
                                                : (const void*)trsm_tc_inv_kernel<TF32>)
                                         : (const void*)trsm_tc_pair_mma_kernel<TF32>;
  return cudaOccupancyMaxActiveClusters(out, fn, &cfg);
}

cudaError_t query_clusters(bool tf32, TileMode mode, int num_sms, int* out, bool f16) {
  return tf32 ? clusters_of<true>(num_sms, mode, out, false) : clusters_of<false>(num_sms, mode, out, f16);
}

template <bool TF32>
static cudaError_t launch_pair(const TcBatch& b, int max_clusters, cudaStream_t s, TileMode mode, bool f16,
                               int stages) {
  const int ncl = b.ntiles < max_clusters ? b.ntiles : max_clusters;
  cudaLaunchAttribute attr[2];
  cudaLaunchConfig_t cfg = pair_config<TF32>(attr, 2 * ncl, s, mode, stages);
  if (mode == TILES_INVERSE) {  // a programmatic dependent of the cast pre-pass (the kernel waits for it)
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.numAttrs = 2;
  }
  if (mode == TILES_INVERSE && stages == 6) {
    if (f16 && !TF32) return cudaLaunchKernelEx(&cfg, trsm_tc_inv_kernel<false, true, 6>, b);
    return cudaLaunchKernelEx(&cfg, trsm_tc_inv_kernel<TF32, false, 6>, b);
  }
  if (mode == TILES_INVERSE && f16 && !TF32) return cudaLaunchKernelEx(&cfg, trsm_tc_inv_kernel<false, true>, b);
  if (mode == TILES_INVERSE) return cudaLaunchKernelEx(&cfg, trsm_tc_inv_kernel<TF32>, b);
  return cudaLaunchKernelEx(&cfg, trsm_tc_pair_mma_kernel<TF32>, b);
}

cudaError_t launch_solve(bool tf32, TileMode mode, const TcBatch& b, int num_sms, int max_clusters,
                         cudaStream_t s, bool f16, int stages) {
  if (f16 && (tf32 || mode != TILES_INVERSE)) return cudaErrorInvalidValue;
  if (mode != TILES_SINGLE && mode != TILES_PAIR_MMA && mode != TILES_INVERSE) return cudaErrorInvalidValue;
  if (stages != 6 && stages != 8) return cudaErrorInvalidValue;
  if (mode != TILES_SINGLE) {
    const cudaError_t e = tf32 ? launch_pair<true>(b, max_clusters, s, mode, false, stages)
                               : launch_pair<false>(b, max_clusters, s, mode, f16, stages);
    return e != cudaSuccess ? e : cudaGetLastError();
  }
  const int grid = b.ntiles < num_sms ? b.ntiles : num_sms;
  if (tf32)
    trsm_tc_kernel<true><<<grid, THREADS, Cfg<true>::SMEM, s>>>(b);
  else
    trsm_tc_kernel<false><<<grid, THREADS, Cfg<false>::SMEM, s>>>(b);
  return cudaGetLastError();
}

}  // namespace tc
}  // namespace gwas
