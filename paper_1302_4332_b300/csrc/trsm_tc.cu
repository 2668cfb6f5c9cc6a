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

#include <algorithm>
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
// K-blocks accumulated in one TMEM partial before the epilogue promotes it:
// one (two measured no faster and raised the error of se up to tenfold); with
// one, all tile modes give the same results bit for bit
constexpr int PROMOTE = 1;

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
  static constexpr int NBARS = 2 * STAGES + 4 + 3 * TRING + 3;
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
  CUtensorMap BhiH, BloH, X8H;  // half-width boxes (128 SNP columns) for the pair modes
  CUtensorMap StX, StHi, StLo;  // pair product's epilogue stores: FP32 X~, hi piece (BF16), lo piece
  CUtensorMap BinHi, BinLo;     // transpose solve: X~ pieces of the forward solve (its diagonal-block input)
  CUtensorMap XcH;              // inverse form: the cast block x - c_i (BF16/FP32), half-width boxes
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
  int pieces;                 // inverse form: also store the hi/lo pieces of X~ (the adjoint's input)
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
  KB_SHARED = 1,  // pair mode, j < 2u: each CTA loads its own Aop and half of X~_jc for both
  KB_LOCAL = 2,   // Aop and all of X~_jc by this CTA alone
  KB_NULL = 3,    // no loads, no MMA: keeps the two CTAs' stage rings in step
  KB_DIAG_IN = 4  // transpose solve, j == k: B = the forward solve's X~ pieces by TMA (3 products)
};

// A work unit.  Single mode: the tile (k, c).  Pair mode: the tiles (2u, c)
// and (2u+1, c) on the two CTAs of a cluster (rank r takes row panel 2u + r).
struct Unit {
  int k;        // this CTA's row panel
  bool has;     // this CTA has a tile (the last unit of an odd P has one)
  bool paired;  // both CTAs have a tile
  int nkb;      // K-blocks in the unit's stage sequence (the same on both CTAs)
};

// UPPER (transpose solve X^ = L^-T X~, single CTAs): row panels from the
// last one up; tile (k, c) walks j = k (its own X~ input), then P-1 .. k+1.
template <bool PAIR, bool UPPER = false>
__device__ __forceinline__ Unit make_unit(int row, const TcStudy& S, uint32_t rank) {
  Unit u;
  if (UPPER) {
    u.k = S.P - 1 - row;
    u.has = true;
    u.paired = false;
    u.nkb = S.P - u.k;
  } else if (PAIR) {
    u.k = 2 * row + (int)rank;
    u.has = u.k < S.P;
    u.paired = 2 * row + 1 < S.P;
    u.nkb = 2 * row + (u.paired ? 2 : 1);
  } else {
    u.k = row;
    u.has = true;
    u.paired = false;
    u.nkb = row + 1;
  }
  return u;
}

// K-block jj of a unit: its kind, and j, the block column of Aop it multiplies.
// Pair mode, both tiles present: rank 0 runs [diag 2u, shared 0..2u-1, null],
// rank 1 [diag 2u+1, shared 0..2u-1, local 2u] (X~ of rank 0's own tile).
template <bool PAIR, bool UPPER = false>
__device__ __forceinline__ KbKind kb_kind(const Unit& u, int row, uint32_t rank, int jj, int& j) {
  if (UPPER) {
    j = jj == 0 ? u.k : u.k + u.nkb - jj;  // k, then P-1 .. k+1
    return jj == 0 ? KB_DIAG_IN : KB_LOCAL;
  }
  if (jj == 0) {
    j = u.k;
    return u.has ? KB_DIAG : KB_NULL;
  }
  if (!PAIR) {
    j = jj - 1;
    return KB_LOCAL;
  }
  if (jj <= 2 * row) {
    j = jj - 1;
    if (u.paired) return KB_SHARED;
    return rank == 0 ? KB_LOCAL : KB_NULL;
  }
  j = 2 * row;
  return rank == 1 ? KB_LOCAL : KB_NULL;
}

template <bool TF32, bool PAIR, bool UPPER = false>
__global__ void __launch_bounds__(THREADS, 1)
    trsm_tc_kernel(const __grid_constant__ TcBatch b) {
  static_assert(!(PAIR && UPPER), "the transpose solve runs on single CTAs");
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
  uint64_t* peer_free = drain + 1;  // pair mode, rank 0: rank 1 is done with a tile-ring slot
  int* tile_ring = reinterpret_cast<int*>(peer_free + TRING);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tile_ring + TRING);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = b.ntiles;  // work units
  DevStatus* st = b.st;
  const uint32_t rank = PAIR ? ptx::cluster_ctarank() : 0u;
  constexpr uint16_t BOTH = 3;  // multicast mask: both CTAs of the pair

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      ptx::mbar_init(&full[s], 2);             // producer (+tx) and producer-or-cast
      ptx::mbar_init(&empty[s], PAIR ? 2 : 1);  // the MMA commit of every CTA that reads the stage
    }
    for (int a = 0; a < 2; ++a) {
      ptx::mbar_init(&part_full[a], 1);           // MMA commit
      ptx::mbar_init(&part_empty[a], EPI_WARPS);  // one arrival per epilogue warp
    }
    for (int i = 0; i < TRING; ++i) {
      ptx::mbar_init(&tile_full[i], 1);
      ptx::mbar_init(&tile_empty[i], 1 + 2 + EPI_WARPS);  // MMA + cast warps + epilogue warps
      ptx::mbar_init(&peer_free[i], 1);
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
      if (PAIR) {
        ptx::prefetch_tensormap(&b.maps[q].BhiH);
        ptx::prefetch_tensormap(&b.maps[q].BloH);
      }
    }
  }
  if (warp == 2) {
    ptx::tmem_alloc(tmem_slot, 2 * TN);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  if (PAIR) ptx::cluster_sync();  // the peer's barriers exist before any remote access
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
        if (!PAIR || rank == 0) {
          // pair mode: rank 0 takes the unit for both CTAs and writes it into
          // rank 1's ring as well, once rank 1 has released the slot
          if (PAIR && !ptx::mbar_wait(&peer_free[slot], use & 1, st)) break;
          t = ptx::aborting(st) ? ntiles : (int)atomicAdd(b.counter, 1u);
          if (t > ntiles) t = ntiles;
          tile_ring[slot] = t;
          if (PAIR) ptx::st_peer_u32(ptx::peer_addr(&tile_ring[slot], 1), (uint32_t)t);
          ptx::mbar_arrive(&tile_full[slot]);
          if (PAIR) ptx::mbar_arrive_peer(ptx::peer_addr(&tile_full[slot], 1));
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
        const Unit u = make_unit<PAIR, UPPER>(row, S, rank);
        if (u.has && !UPPER) {
          if (!ptx::mbar_wait(x8_empty, (x8n & 1) ^ 1, st)) break;
          ptx::mbar_arrive_expect_tx(x8_full, K::X8_BYTES);
          ptx::tma_load_2d(x8, &M.X8, x8_full, u.k * TB, c * TN);
          ++x8n;
        }
        bool ok = true;
        for (int jj = 0; jj < u.nkb && ok; ++jj) {
          int j;
          const KbKind kind = kb_kind<PAIR, UPPER>(u, row, rank, jj, j);
          if (kind == KB_SHARED || kind == KB_LOCAL) {
            if (!ptx::wait_flag(&S.flags[j * S.C + c], st)) { ok = false; break; }
            ptx::fence_proxy_async_global();
          }
          for (int h = 0; h < K::CPB; ++h, ++cnt) {
            const int s = cnt % STAGES;
            const uint32_t r = cnt / STAGES;
            if (!ptx::mbar_wait(&empty[s], (r & 1) ^ 1, st)) { ok = false; break; }
            uint8_t* sb = smem + s * K::STAGE_BYTES;
            const int kx = j * TB + h * K::KCH;
            if (kind == KB_NULL) {
              ptx::mbar_arrive(&full[s]);
              ptx::mbar_arrive(&full[s]);
            } else if (kind == KB_DIAG) {
              ptx::mbar_arrive_expect_tx(&full[s], 2 * K::A_BYTES);
              ptx::tma_load_2d(sb, &M.Ahi, &full[s], kx, u.k * TB);
              ptx::tma_load_2d(sb + K::A_BYTES, &M.Alo, &full[s], kx, u.k * TB);
            } else {
              ptx::mbar_arrive_expect_tx(&full[s], 2 * K::A_BYTES + 2 * K::B_BYTES);
              ptx::tma_load_2d(sb, &M.Ahi, &full[s], kx, u.k * TB);
              ptx::tma_load_2d(sb + K::A_BYTES, &M.Alo, &full[s], kx, u.k * TB);
              if (PAIR && kind == KB_SHARED) {
                // this CTA's half of the strip's columns, into both CTAs (the
                // peer sends the other half); the 8 KB offset keeps the
                // 512-byte swizzle atoms of a full-width load
                constexpr int HB = K::B_BYTES / 2;
                const int y = c * TN + (int)rank * (TN / 2);
                ptx::tma_load_2d_mc(sb + 2 * K::A_BYTES + rank * HB, &M.BhiH, &full[s], kx, y, BOTH);
                ptx::tma_load_2d_mc(sb + 2 * K::A_BYTES + K::B_BYTES + rank * HB, &M.BloH, &full[s], kx, y, BOTH);
              } else if (UPPER && kind == KB_DIAG_IN) {
                ptx::tma_load_2d(sb + 2 * K::A_BYTES, &M.BinHi, &full[s], kx, c * TN);
                ptx::tma_load_2d(sb + 2 * K::A_BYTES + K::B_BYTES, &M.BinLo, &full[s], kx, c * TN);
              } else {
                ptx::tma_load_2d(sb + 2 * K::A_BYTES, &M.Bhi, &full[s], kx, c * TN);
                ptx::tma_load_2d(sb + 2 * K::A_BYTES + K::B_BYTES, &M.Blo, &full[s], kx, c * TN);
              }
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
      // a consumed stage is released to every CTA that writes it
      auto release = [&](int s) {
        if (PAIR)
          ptx::mma_commit_mc(&empty[s], BOTH);
        else
          ptx::mma_commit(&empty[s]);
      };
      for (int it = 0;; ++it) {
        const int slot = it % TRING;
        const uint32_t use = it / TRING;
        if (!ptx::mbar_wait_s<PAIR>(&tile_full[slot], use & 1, st)) break;
        const int t = tile_ring[slot];
        ptx::mbar_arrive(&tile_empty[slot]);
        if (t >= ntiles) break;
        int sidx, row, c;
        TcStudy S;
        decode_tile(b, t, sidx, row, c, S);
        const Unit u = make_unit<PAIR, UPPER>(row, S, rank);
        bool ok = true;
        int q = 0;  // K-blocks of this CTA's tile issued so far (k + 1 in all)
        int a = 0;
        uint32_t d = 0, accumulate = 0;
        for (int jj = 0; jj < u.nkb && ok; ++jj) {
          int j;
          const KbKind kind = kb_kind<PAIR, UPPER>(u, row, rank, jj, j);
          if (kind == KB_NULL) {
            for (int h = 0; h < K::CPB; ++h, ++cnt) {
              const int s = cnt % STAGES;
              if (!ptx::mbar_wait(&full[s], (cnt / STAGES) & 1, st)) { ok = false; break; }
              release(s);
            }
            continue;
          }
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
          const int nk = UPPER ? u.nkb : u.k + 1;  // the tile's K-blocks
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
      if (!ptx::group_and(2, 64, ptx::mbar_wait_s<PAIR>(&tile_full[slot], use & 1, st))) break;
      const int t = tile_ring[slot];
      ptx::named_bar(2, 64);
      if (lane == 0) ptx::mbar_arrive(&tile_empty[slot]);
      if (t >= ntiles) break;
      int sidx, row, ctile;
      TcStudy S;
      decode_tile(b, t, sidx, row, ctile, S);
      const Unit u = make_unit<PAIR, UPPER>(row, S, rank);
      if (u.has && !UPPER) {
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
      if (!ptx::group_and(1, NT, ptx::mbar_wait_s<PAIR>(&tile_full[slot], use & 1, st))) break;
      const int t = tile_ring[slot];
      ptx::named_bar(1, NT);
      if (lane == 0) ptx::mbar_arrive(&tile_empty[slot]);
      if (t >= ntiles) break;
      int sidx, row, c;
      TcStudy S;
      decode_tile(b, t, sidx, row, c, S);
      const Unit u = make_unit<PAIR, UPPER>(row, S, rank);
      if (!u.has) continue;
      const int k = u.k;
#pragma unroll
      for (int i = 0; i < EPI_COLS; ++i) master[i] = 0.f;
      bool ok = true;
      const int nk = UPPER ? u.nkb : k + 1;  // the tile's K-blocks
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
  // pair mode: neither CTA retires while the other may still write its shared
  // memory or arrive on its barriers
  if (PAIR) ptx::cluster_sync();
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
// SNP columns per 2 KB epilogue store chunk (32 rows): BF16 mode stores hi+lo
// chunks (4 B per element), then FP32 chunks; TF32 mode FP32+lo chunks (8 B)
template <bool TF32>
constexpr int st_cols() { return TF32 ? 8 : 16; }

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
constexpr int STAGES = 8;
constexpr int ST_COLS = 16;  // SNP columns per epilogue store chunk (32 rows x 16 FP32 = 2 KB)

template <bool TF32>
struct Cfg {
  static constexpr int ESZ = TF32 ? 4 : 2;
  static constexpr int KCH = 64 / ESZ;
  static constexpr int KMMA = TF32 ? 8 : 16;
  static constexpr int CPB = TB / KCH;
  static constexpr int A_BYTES = TB * 64;                    // one piece of this CTA's L^-1 rows: 8 KB
  static constexpr int B_BYTES = (TN / 2) * 64;              // this CTA's half of the SNP columns: 8 KB
  static constexpr int STAGE_BYTES = 2 * A_BYTES + B_BYTES;  // 24 KB
  static constexpr int CHUNK_BYTES = 2048;
  static constexpr int STG_OFF = STAGES * STAGE_BYTES;
  static constexpr int BAR_OFF = STG_OFF + EPI_WARPS * 2 * CHUNK_BYTES;
  static constexpr int NBARS = 2 * STAGES + 4 + 3 * TRING + 1;
  static constexpr int SMEM = 1024 + BAR_OFF + NBARS * 8 + TRING * 4 + 16;
  static_assert(SMEM <= 232448, "shared memory per CTA");
};
}  // namespace inv2

template <bool TF32>
__global__ void __launch_bounds__(THREADS, 1) trsm_tc_inv_kernel(const __grid_constant__ TcBatch b) {
  using K = inv2::Cfg<TF32>;
  constexpr int ST = inv2::STAGES;
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
        if (t >= ntiles) break;
        int sidx, row, c;
        TcStudy S;
        decode_tile(b, t, sidx, row, c, S);
        const TcMaps& M = b.maps[sidx];
        const pair2::Unit u = pair2::make_unit(row, S);
        const int arow = rank == 0 ? u.k0 : (u.paired ? u.k0 + 1 : -1);  // this CTA's row panel
        const int ycol = c * TN + (int)rank * (TN / 2);                   // this CTA's SNP columns
        bool ok = true;
        for (int j = 0; j < u.nkb && ok; ++j) {
          // block (arow, j) above the diagonal, or no rows: a box wholly outside reads zeros
          const int ay = (arow >= 0 && j <= arow) ? arow * TB : -TB;
          for (int h = 0; h < K::CPB; ++h, ++cnt) {
            const int s = cnt % ST;
            const uint32_t r = cnt / ST;
            if (!ptx::mbar_wait(&empty[s], (r & 1) ^ 1, st)) { ok = false; break; }
            uint8_t* sb = smem + s * K::STAGE_BYTES;
            const int kx = j * TB + h * K::KCH;
            const uint32_t fb = lead_addr(&full[s]);
            if (leader)
              ptx::mbar_arrive_expect_tx(&full[s], 2 * K::STAGE_BYTES);
            else
              ptx::mbar_arrive_peer_count(fb);
            ptx::tma_load_2d_pair(sb, &M.Ahi, fb, kx, ay);
            ptx::tma_load_2d_pair(sb + K::A_BYTES, &M.Alo, fb, kx, ay);
            ptx::tma_load_2d_pair(sb + 2 * K::A_BYTES, &M.XcH, fb, kx, ycol);
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
        for (int j = 0; j < u.nkb && ok; ++j) {
          // every K-block into a fresh partial (promoted by the epilogue)
          const int a = kb & 1;
          if (!ptx::mbar_wait(&part_empty[a], ((kb >> 1) & 1) ^ 1, st)) { ok = false; break; }
          ++kb;
          ptx::tc_fence_after();
          const uint32_t d = tmem_base + a * TN;
          uint32_t accumulate = 0;
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
              const uint64_t bx = ptx::sdesc_k64(base + 2 * K::A_BYTES + off);
              ptx::mma_pair<TF32>(d, alo, bx, idesc, accumulate);
              accumulate = 1;
              ptx::mma_pair<TF32>(d, ahi, bx, idesc, 1);
            }
            ptx::mma_commit_pair(&empty[s], BOTH);
          }
          if (!ok) break;
          ptx::mma_commit_pair(&part_full[a], BOTH);
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
      const pair2::Unit u = pair2::make_unit(row, S);
      const bool has = leader || u.paired;  // this CTA has a tile
      const int k = u.k0 + (int)rank;
#pragma unroll
      for (int i = 0; i < EPI_COLS; ++i) master[i] = 0.f;
      bool ok = true;
      for (int pp = 0; pp < u.nkb && ok; ++pp) {
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
      // X~ of this CTA's tile to HBM by TMA stores of shared-memory chunks (and,
      // for the transpose solve of the adjoint form, its hi/lo pieces)
      const TcMaps& M = b.maps[sidx];
      uint8_t* stg = smem + K::STG_OFF + e * 2 * K::CHUNK_BYTES;
      const int r0 = k * TB + 32 * lq;
      const int c0 = c * TN + chalf * EPI_COLS;
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
      if (b.pieces) {
#pragma unroll
        for (int q = 0; q < EPI_COLS / CC; ++q) {
          uint8_t* buf = next_buf();
#pragma unroll
          for (int i = 0; i < CC; ++i) {
            const float x = master[q * CC + i];
            if constexpr (TF32) {
              reinterpret_cast<float*>(buf)[i * 32 + lane] = x - __uint_as_float(tf32_trunc_bits(x));
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
            if constexpr (TF32) {
              ptx::tma_store_2d(&M.StLo, buf, r0, c0 + q * CC);
            } else {
              ptx::tma_store_2d(&M.StHi, buf, r0, c0 + q * CC);
              ptx::tma_store_2d(&M.StLo, buf + 1024, r0, c0 + q * CC);
            }
            ptx::bulk_commit();
          }
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

// B operand of the inverse form: x'_ri = x_ri - c_i on rows < n and 0 on rows
// n..n_pad-1, as BF16 (or FP32, read as TF32 by the tensor cores), column-major
// with leading dimension n_pad.  c_i is computed here as in column_shift_kernel
// when `shift` is given (and stored there), else 0.  One warp per SNP column.
template <bool TF32>
__global__ void cast_shift_kernel(const int8_t* __restrict__ X, int64_t ldx, int n, int n_pad, int ncols,
                                  int8_t* __restrict__ shift, void* __restrict__ xc) {
  const int lane = threadIdx.x & 31;
  const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (col >= ncols) return;
  const int8_t* x = X + (int64_t)col * ldx;  // 16-byte aligned (checked by the caller)
  const int n16 = n & ~15;
  int c = 0;
  if (shift) {
    int sum = 0;
    for (int r = lane * 16; r < n16; r += 32 * 16) {
      const int4 v = __ldg(reinterpret_cast<const int4*>(x + r));
      const int w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) sum += __dp4a(w[i], 0x01010101, 0);
    }
    for (int r = n16 + lane; r < n; r += 32) sum += x[r];
#pragma unroll
    for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    const long long num = 2LL * sum + n, den = 2LL * n;
    long long cc = num >= 0 ? num / den : -((-num + den - 1) / den);
    cc = cc > 127 ? 127 : (cc < -127 ? -127 : cc);
    c = (int)cc;
    if (lane == 0) shift[col] = (int8_t)c;
  }
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
    if constexpr (TF32) {
      float4* o = reinterpret_cast<float4*>(static_cast<float*>(xc) + (int64_t)col * n_pad + r);
#pragma unroll
      for (int i = 0; i < 4; ++i) o[i] = make_float4(f[4 * i], f[4 * i + 1], f[4 * i + 2], f[4 * i + 3]);
    } else {
      uint32_t wv[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const __nv_bfloat162 b2 = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
        wv[i] = *reinterpret_cast<const uint32_t*>(&b2);
      }
      uint4* o = reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(xc) + (int64_t)col * n_pad + r);
      o[0] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
      o[1] = make_uint4(wv[4], wv[5], wv[6], wv[7]);
    }
  }
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

// Columns c0.. of L^-1, solved into `xt` (FP32, column-major, leading
// dimension ldt), transposed into the row-major hi/lo pieces of the inverse
// form's operator.  Entries above the diagonal and in the padding rows and
// columns (index >= n) are set to zero.  32 x 32 tiles through shared memory.
template <bool TF32>
__global__ void linv_split_kernel(const float* __restrict__ xt, int64_t ldt, int n, int n_pad, int c0, int ncols,
                                  void* __restrict__ hi, void* __restrict__ lo) {
  __shared__ float tile[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  const int q0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int q = q0 + ty + 8 * i;
    tile[ty + 8 * i][tx] = q < ncols ? xt[(int64_t)q * ldt + r0 + tx] : 0.f;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int row = r0 + ty + 8 * i, q = q0 + tx, gcol = c0 + q;
    if (q >= ncols) continue;
    float v = tile[tx][ty + 8 * i];
    if (row >= n || gcol >= n || gcol > row) v = 0.f;
    const int64_t idx = (int64_t)row * n_pad + gcol;
    if constexpr (TF32) {
      uint32_t hb;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hb) : "f"(v));
      const float h = __uint_as_float(hb);
      static_cast<float*>(hi)[idx] = h;
      static_cast<float*>(lo)[idx] = v - h;
    } else {
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      static_cast<__nv_bfloat16*>(hi)[idx] = h;
      static_cast<__nv_bfloat16*>(lo)[idx] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
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
  TileMode mode = TILES_SINGLE;    // how tiles map onto CTAs
  int max_clusters = 0;            // pair modes: co-resident 2-CTA clusters of the kernel
  uint32_t* order = nullptr;      // device tile order when strip_group > 0
  TcStudy* study_dev = nullptr;   // device copy of the study descriptor (grouped order)
  int order_C = -1;               // the column-strip count the order was built for
  unsigned int* sched = nullptr;  // [0] counter, flags from +32
  size_t sched_bytes = 0;
  DevStatus* st = nullptr;
  CUtensorMap mAhi, mAlo, mBhi, mBlo, mBhiH, mBloH;
  CUtensorMap mStX, mStHi, mStLo;  // pair product's epilogue stores
  // transpose solve (the adjoint form): the transpose block operator split hi/lo,
  // X^ = L^-T X~ in FP32 + pieces, and their maps
  void* ahiT = nullptr;
  void* aloT = nullptr;
  float* xh32 = nullptr;
  void* xhhi = nullptr;
  void* xhlo = nullptr;
  CUtensorMap mAhiT, mAloT, mBhiT, mBloT;
  void* xc = nullptr;  // inverse form: the cast block x - c_i (n_pad x bs, BF16 or FP32)
  EncodeTiledFn encode = nullptr;
};

// Row entries of the tile order: row panels, or row-panel pairs in pair mode.
static int unit_rows(const TcState* t) { return t->mode == TILES_SINGLE ? t->P : (t->P + 1) / 2; }

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

template <bool TF32, bool PAIR>
static cudaError_t set_smem_attr() {
  return cudaFuncSetAttribute(trsm_tc_kernel<TF32, PAIR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              Cfg<TF32>::SMEM);
}

template <bool TF32>
static cudaError_t set_smem_attr_upper() {
  return cudaFuncSetAttribute(trsm_tc_kernel<TF32, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              Cfg<TF32>::SMEM);
}

template <bool TF32>
static cudaError_t set_smem_attr_pair_mma() {
  return cudaFuncSetAttribute(trsm_tc_pair_mma_kernel<TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              pair2::Cfg<TF32>::SMEM);
}

template <bool TF32>
static cudaError_t set_smem_attr_inv() {
  return cudaFuncSetAttribute(trsm_tc_inv_kernel<TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              inv2::Cfg<TF32>::SMEM);
}

template <bool TF32>
static cudaLaunchConfig_t pair_config(cudaLaunchAttribute* attr, int grid, cudaStream_t s, TileMode mode) {
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof cfg);
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(THREADS);
  cfg.dynamicSmemBytes = mode == TILES_INVERSE    ? inv2::Cfg<TF32>::SMEM
                         : mode == TILES_PAIR_MMA ? pair2::Cfg<TF32>::SMEM
                                                  : Cfg<TF32>::SMEM;
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

// Co-resident 2-CTA clusters of a pair kernel (one CTA per SM).
template <bool TF32>
static cudaError_t query_clusters(int num_sms, TileMode mode, int* out) {
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = pair_config<TF32>(attr, 2 * (num_sms / 2), nullptr, mode);
  const void* fn = mode == TILES_INVERSE    ? (const void*)trsm_tc_inv_kernel<TF32>
                   : mode == TILES_PAIR_MMA ? (const void*)trsm_tc_pair_mma_kernel<TF32>
                                            : (const void*)trsm_tc_kernel<TF32, true>;
  return cudaOccupancyMaxActiveClusters(out, fn, &cfg);
}

static cudaError_t build_inverse(TcState* t, const double* Aop, cudaStream_t s, int64_t* launches);

cudaError_t create(TcState** out, Split split, const double* Aop, int n, int n_pad, int bs, int num_sms,
                   bool center, DevStatus* st, cudaStream_t s, int64_t* launches, int strip_group, TileMode mode) {
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
  // measured at n = 1e4 with 4096-column blocks: the inverse form is the
  // fastest for both splits (BF16: 0.51 ms a block against 0.93 ms for the
  // pair product of the substitution)
  if (mode == TILES_AUTO) mode = TILES_INVERSE;
  t->mode = mode;
  const bool inv = mode == TILES_INVERSE;
  if (inv) TRY(cudaMalloc(&t->xc, esz * (size_t)n_pad * bs));
  if (strip_group > 0 || inv) {
    TRY(cudaMalloc(&t->order, sizeof(uint32_t) * (size_t)t->P * Cmax));
    TRY(cudaMalloc(&t->study_dev, sizeof(TcStudy)));
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
  const uint32_t kch = t->tf32 ? Cfg<true>::KCH : Cfg<false>::KCH;
  TRY(make_map(t->encode, &t->mAhi, dt, t->ahi, n_pad, n_pad, esz * n_pad, kch, TB, true));
  TRY(make_map(t->encode, &t->mAlo, dt, t->alo, n_pad, n_pad, esz * n_pad, kch, TB, true));
  const void* bhi_base = t->tf32 ? static_cast<const void*>(t->xt32) : t->bhi;
  TRY(make_map(t->encode, &t->mBhi, dt, bhi_base, n_pad, bs, esz * n_pad, kch, TN, true));
  TRY(make_map(t->encode, &t->mBlo, dt, t->blo, n_pad, bs, esz * n_pad, kch, TN, true));
  TRY(make_map(t->encode, &t->mBhiH, dt, bhi_base, n_pad, bs, esz * n_pad, kch, TN / 2, true));
  TRY(make_map(t->encode, &t->mBloH, dt, t->blo, n_pad, bs, esz * n_pad, kch, TN / 2, true));
  // epilogue store chunks: the pair product's (value + pieces in one 2 KB
  // buffer), or the inverse form's (FP32 value alone, 16 columns)
  const uint32_t stc = inv ? inv2::ST_COLS : (t->tf32 ? pair2::st_cols<true>() : pair2::st_cols<false>());
  TRY(make_map(t->encode, &t->mStX, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, t->xt32, n_pad, bs, 4 * (size_t)n_pad, 32, stc,
               false));
  memset(&t->mStHi, 0, sizeof t->mStHi);
  if (!t->tf32) TRY(make_map(t->encode, &t->mStHi, dt, t->bhi, n_pad, bs, esz * n_pad, 32, stc, false));
  TRY(make_map(t->encode, &t->mStLo, dt, t->blo, n_pad, bs, esz * n_pad, 32, stc, false));
  TRY((t->tf32 ? set_smem_attr<true, false>() : set_smem_attr<false, false>()));
  if (mode != TILES_SINGLE) {
    TRY((t->tf32 ? set_smem_attr<true, true>() : set_smem_attr<false, true>()));
    TRY((t->tf32 ? set_smem_attr_pair_mma<true>() : set_smem_attr_pair_mma<false>()));
    TRY((t->tf32 ? set_smem_attr_inv<true>() : set_smem_attr_inv<false>()));
    TRY((t->tf32 ? query_clusters<true>(num_sms, mode, &t->max_clusters)
                 : query_clusters<false>(num_sms, mode, &t->max_clusters)));
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
static void append_units(std::vector<UnitKey>& v, int si, int P, int C) {
  for (int r = 0; r < (P + 1) / 2; ++r) {
    const int len = 2 * r + (2 * r + 1 < P ? 2 : 1);
    for (int c = 0; c < C; ++c) v.push_back({len, ((uint32_t)si << 28) | ((uint32_t)r << 14) | (uint32_t)c});
  }
}
static void longest_first(std::vector<UnitKey>& v, std::vector<uint32_t>& order) {
  std::stable_sort(v.begin(), v.end(), [](const UnitKey& a, const UnitKey& b) { return a.len > b.len; });
  for (const UnitKey& u : v) order.push_back(u.code);
}

// Inverse form: the cast block's map (half-width boxes) and the cast
// pre-pass (with the integer shifts when centering).
static cudaError_t prepare_cast(TcState* t, const int8_t* X, int64_t ldx, int ncols, cudaStream_t s,
                                int64_t* launches, CUtensorMap* mXcH) {
  const size_t esz = t->tf32 ? 4 : 2;
  const CUtensorMapDataType dt = t->tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const uint32_t kch = t->tf32 ? Cfg<true>::KCH : Cfg<false>::KCH;
  cudaError_t e = make_map(t->encode, mXcH, dt, t->xc, (uint64_t)t->n_pad, (uint64_t)ncols, esz * t->n_pad, kch,
                           TN / 2, true);
  if (e != cudaSuccess) return e;
  int8_t* sh = t->center ? t->shift : nullptr;
  if (t->tf32)
    cast_shift_kernel<true><<<(ncols + 7) / 8, 256, 0, s>>>(X, ldx, t->n, t->n_pad, ncols, sh, t->xc);
  else
    cast_shift_kernel<false><<<(ncols + 7) / 8, 256, 0, s>>>(X, ldx, t->n, t->n_pad, ncols, sh, t->xc);
  ++*launches;
  return cudaGetLastError();
}

// The study part of one launch: int8 map, cleared flags, integer shifts.
static cudaError_t prepare_study(TcState* t, const int8_t* X, int64_t ldx, int ncols, cudaStream_t s,
                                 int64_t* launches, TcStudy* S, CUtensorMap* mX8, CUtensorMap* mX8H,
                                 CUtensorMap* mXcH) {
  if (ncols > t->bs || (reinterpret_cast<uintptr_t>(X) & 15) || (ldx & 15) || ldx < t->n)
    return cudaErrorInvalidValue;
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
  e = cudaMemsetAsync(t->sched, 0, 128 + sizeof(int) * (size_t)t->P * C, s);
  if (e != cudaSuccess) return e;
  if (t->mode == TILES_INVERSE) {
    if ((e = prepare_cast(t, X, ldx, ncols, s, launches, mXcH)) != cudaSuccess) return e;
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
  return cudaSuccess;
}

template <bool TF32>
static cudaError_t launch_pair(const TcBatch& b, int max_clusters, cudaStream_t s, TileMode mode) {
  const int ncl = b.ntiles < max_clusters ? b.ntiles : max_clusters;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = pair_config<TF32>(attr, 2 * ncl, s, mode);
  if (mode == TILES_INVERSE) return cudaLaunchKernelEx(&cfg, trsm_tc_inv_kernel<TF32>, b);
  if (mode == TILES_PAIR_MMA) return cudaLaunchKernelEx(&cfg, trsm_tc_pair_mma_kernel<TF32>, b);
  return cudaLaunchKernelEx(&cfg, trsm_tc_kernel<TF32, true>, b);
}

// b.ntiles work units: tiles, or (pair modes) row-panel pairs of a strip.
static cudaError_t launch_kernel(bool tf32, TileMode mode, const TcBatch& b, int num_sms, int max_clusters,
                                 cudaStream_t s, int64_t* launches) {
  ++*launches;
  if (mode != TILES_SINGLE) {
    const cudaError_t e =
        tf32 ? launch_pair<true>(b, max_clusters, s, mode) : launch_pair<false>(b, max_clusters, s, mode);
    return e != cudaSuccess ? e : cudaGetLastError();
  }
  const int grid = b.ntiles < num_sms ? b.ntiles : num_sms;
  if (tf32)
    trsm_tc_kernel<true, false><<<grid, THREADS, Cfg<true>::SMEM, s>>>(b);
  else
    trsm_tc_kernel<false, false><<<grid, THREADS, Cfg<false>::SMEM, s>>>(b);
  return cudaGetLastError();
}

cudaError_t run_block(TcState* t, const int8_t* X, int64_t ldx, int ncols, cudaStream_t s, int64_t* launches,
                      bool pieces) {
  if (ncols <= 0) return cudaSuccess;
  TcBatch b;
  memset(&b, 0, sizeof b);
  cudaError_t e =
      prepare_study(t, X, ldx, ncols, s, launches, &b.s0, &b.maps[0].X8, &b.maps[0].X8H, &b.maps[0].XcH);
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
  b.pieces = pieces ? 1 : 0;
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
    // the grouped order reads the study descriptor from device memory
    if ((e = cudaMemcpyAsync(t->study_dev, &b.s0, sizeof(TcStudy), cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
    b.order = t->order;
    b.studies = t->study_dev;
  }
  return launch_kernel(t->tf32, t->mode, b, t->num_sms, t->max_clusters, s, launches);
}

// Inverse form set-up: L^-1 = the substitution applied to the identity, on
// the tensor cores in TF32x3 (the pair product over Aop, 4096 identity
// columns per launch, no centering), then transposed and split into the
// row-major hi/lo pieces of t.  Synchronizes the stream.
static cudaError_t build_inverse(TcState* t, const double* Aop, cudaStream_t s, int64_t* launches) {
  const int np = t->n_pad;
  const int bsi = np < 4096 ? np : 4096;
  TcState* g = nullptr;
  cudaError_t e = create(&g, SPLIT_TF32, Aop, t->n, np, bsi, t->num_sms, false, t->st, s, launches, 0, TILES_PAIR_MMA);
  if (e != cudaSuccess) return e;
  int8_t* eye = nullptr;
  e = cudaMalloc(&eye, (size_t)np * bsi);
  for (int c0 = 0; e == cudaSuccess && c0 < np; c0 += bsi) {
    const int nc = np - c0 < bsi ? np - c0 : bsi;
    identity_i8_kernel<<<1184, 256, 0, s>>>(eye, np, c0, nc);
    ++*launches;
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((e = run_block(g, eye, np, nc, s, launches)) != cudaSuccess) break;
    const dim3 grid((nc + 31) / 32, np / 32);
    if (t->tf32)
      linv_split_kernel<true><<<grid, dim3(32, 8), 0, s>>>(g->xt32, g->ldt, t->n, np, c0, nc, t->ahi, t->alo);
    else
      linv_split_kernel<false><<<grid, dim3(32, 8), 0, s>>>(g->xt32, g->ldt, t->n, np, c0, nc, t->ahi, t->alo);
    ++*launches;
    e = cudaGetLastError();
  }
  const cudaError_t es = cudaStreamSynchronize(s);  // before g's buffers go
  if (e == cudaSuccess) e = es;
  if (e == cudaSuccess && t->st) {
    DevStatus h;
    if ((e = cudaMemcpy(&h, t->st, sizeof h, cudaMemcpyDeviceToHost)) == cudaSuccess && h.err != DEV_OK)
      e = cudaErrorLaunchTimeout;  // a bounded wait of the solve expired
  }
  cudaFree(eye);
  destroy(g);
  return e;
}

// ------------------------------------------------------ transpose solve (adjoint)
cudaError_t ensure_transpose(TcState* t, const double* AopT, cudaStream_t s, int64_t* launches) {
  if (t->ahiT) return cudaSuccess;
  const size_t esz = t->tf32 ? 4 : 2;
  const size_t np = (size_t)t->n_pad, n2 = np * np;
  cudaError_t e;
  if ((e = cudaMalloc(&t->ahiT, esz * n2)) != cudaSuccess || (e = cudaMalloc(&t->aloT, esz * n2)) != cudaSuccess ||
      (e = cudaMalloc(&t->xh32, sizeof(float) * np * t->bs)) != cudaSuccess ||
      (!t->tf32 && (e = cudaMalloc(&t->xhhi, 2 * np * t->bs)) != cudaSuccess) ||
      (e = cudaMalloc(&t->xhlo, esz * np * t->bs)) != cudaSuccess)
    return e;
  if (t->tf32)
    split_aop_kernel<true><<<1184, 256, 0, s>>>(AopT, (int64_t)n2, t->ahiT, t->aloT);
  else
    split_aop_kernel<false><<<1184, 256, 0, s>>>(AopT, (int64_t)n2, t->ahiT, t->aloT);
  ++*launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const CUtensorMapDataType dt = t->tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const uint32_t kch = t->tf32 ? Cfg<true>::KCH : Cfg<false>::KCH;
  const void* bhi = t->tf32 ? static_cast<const void*>(t->xh32) : t->xhhi;
  if ((e = make_map(t->encode, &t->mAhiT, dt, t->ahiT, np, np, esz * np, kch, TB, true)) != cudaSuccess ||
      (e = make_map(t->encode, &t->mAloT, dt, t->aloT, np, np, esz * np, kch, TB, true)) != cudaSuccess ||
      (e = make_map(t->encode, &t->mBhiT, dt, bhi, np, t->bs, esz * np, kch, TN, true)) != cudaSuccess ||
      (e = make_map(t->encode, &t->mBloT, dt, t->xhlo, np, t->bs, esz * np, kch, TN, true)) != cudaSuccess)
    return e;
  return t->tf32 ? set_smem_attr_upper<true>() : set_smem_attr_upper<false>();
}

cudaError_t run_transpose(TcState* t, int ncols, cudaStream_t s, int64_t* launches) {
  if (ncols <= 0) return cudaSuccess;
  if (!t->ahiT || ncols > t->bs) return cudaErrorInvalidValue;
  TcBatch b;
  memset(&b, 0, sizeof b);
  const int C = (ncols + TN - 1) / TN;
  cudaError_t e = cudaMemsetAsync(t->sched, 0, 128 + sizeof(int) * (size_t)t->P * C, s);
  if (e != cudaSuccess) return e;
  TcStudy& S = b.s0;
  S.P = t->P;
  S.C = C;
  S.ncols = ncols;
  S.n = t->n;
  S.shift = nullptr;
  S.flags = reinterpret_cast<int*>(t->sched + 32);
  S.xt32 = t->xh32;
  S.bhi = t->xhhi;
  S.blo = t->xhlo;
  S.ldt = t->ldt;
  b.maps[0].Ahi = t->mAhiT;
  b.maps[0].Alo = t->mAloT;
  b.maps[0].Bhi = t->mBhiT;
  b.maps[0].Blo = t->mBloT;
  b.maps[0].BinHi = t->mBhi;  // the forward solve's X~ pieces
  b.maps[0].BinLo = t->mBlo;
  b.nstudies = 1;
  b.ntiles = t->P * C;
  b.counter = t->sched;
  b.st = t->st;
  const int grid = b.ntiles < t->num_sms ? b.ntiles : t->num_sms;
  if (t->tf32)
    trsm_tc_kernel<true, false, true><<<grid, THREADS, Cfg<true>::SMEM, s>>>(b);
  else
    trsm_tc_kernel<false, false, true><<<grid, THREADS, Cfg<false>::SMEM, s>>>(b);
  ++*launches;
  return cudaGetLastError();
}

const float* xhat_f32(const TcState* t) { return t->xh32; }

// ------------------------------------------------------------- batched launch
struct TcBatchState {
  int nstudies = 0;
  int ntiles = 0;
  TcStudy S[MAX_STUDIES];
  CUtensorMap mX8[MAX_STUDIES], mX8H[MAX_STUDIES], mXcH[MAX_STUDIES] = {};
  const int8_t* X[MAX_STUDIES];
  int64_t ldx[MAX_STUDIES];
  bool tf32 = false;
  TileMode mode = TILES_SINGLE;
  int num_sms = 0, max_clusters = 0;
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
    if (ts[i]->tf32 != ts[0]->tf32 || ts[i]->mode != ts[0]->mode) return cudaErrorInvalidValue;
  TcBatchState* B = new TcBatchState;
  B->nstudies = nstudies;
  B->tf32 = ts[0]->tf32;
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
                   t->tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, t->xc,
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
  for (int i = 0; i < B->nstudies; ++i) {
    if (B->S[i].ncols == 0) continue;
    TcState* t = ts[i];
    if ((e = cudaMemsetAsync(t->sched, 0, 128 + sizeof(int) * (size_t)t->P * B->S[i].C, s)) != cudaSuccess) return e;
    if (t->mode == TILES_INVERSE) {
      int8_t* sh = t->center ? t->shift : nullptr;
      const int nc = B->S[i].ncols;
      if (t->tf32)
        cast_shift_kernel<true><<<(nc + 7) / 8, 256, 0, s>>>(B->X[i], B->ldx[i], t->n, t->n_pad, nc, sh, t->xc);
      else
        cast_shift_kernel<false><<<(nc + 7) / 8, 256, 0, s>>>(B->X[i], B->ldx[i], t->n, t->n_pad, nc, sh, t->xc);
      ++*launches;
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
  if ((e = cudaMemsetAsync(B->d_counter, 0, 128, s)) != cudaSuccess) return e;
  b.studies = B->d_studies;
  b.order = B->d_order;
  b.nstudies = B->nstudies;
  b.ntiles = B->ntiles;
  b.counter = B->d_counter;
  b.st = B->st;
  return launch_kernel(B->tf32, B->mode, b, B->num_sms, B->max_clusters, s, launches);
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
  cudaFree(t->ahiT);
  cudaFree(t->aloT);
  cudaFree(t->xh32);
  cudaFree(t->xhhi);
  cudaFree(t->xhlo);
  cudaFree(t->ahi);
  cudaFree(t->alo);
  cudaFree(t->xt32);
  cudaFree(t->bhi);
  cudaFree(t->blo);
  cudaFree(t->xc);
  cudaFree(t->sched);
  cudaFree(t->shift);
  cudaFree(t->order);
  cudaFree(t->study_dev);
  delete t;
}

}  // namespace tc
}  // namespace gwas
