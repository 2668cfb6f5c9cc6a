// Exact integer products of a sliced M^-1 on the tensor cores, in two uses:
// the split precisions' adjoint (a11) and the sliced solve (GWAS_SLICED64, the
// FP64 bar from the tensor cores).
//
// With W = M^-1 (symmetric), X^_L = W X_L, y^ = W y and x' = x - c 1 (the SNP
// column shifted by the integer nearest its mean when X_L[:, 0] is the
// intercept: [X_L | x'] spans the same space, so b_p, its se, the Wald
// statistic and its gradient do not change, and b_0 maps back exactly), the
// per-SNP inputs are products of fixed FP64 data with the small integers x':
//   forward sums    x~^T X~_L = x'^T X^_L,  x~^T y~ = x'^T y^,  x~^T x~ = x'^T (W x'),
//   transpose sums  x^^T X^_L = x'^T (W X^_L),  x^^T y^ = x'^T (W y^),  ||x^||^2 = ||W x'||^2,
// (x~ = L^-1 x', x^ = L^-T x~ = W x': Eq. 1's X_i^T M^-1 X_i and X_i^T M^-1 y
// with M^-1 explicit).  So one product per block, A x':
//   adjoint   A = [ W ; X^_L^T ; y^T ; (W X^_L)^T ; (W y^)^T ],
//   solve     A = [ T ; X^_L^T ; Y^^T ],  T = W's lower triangle with its diagonal
//             halved (x'^T W x' = 2 x'^T T x'), so that the product skips the
//             K-blocks above each row pair's diagonal;
// the arithmetic after the product (adjoint.cu, reduce_solve.cu) is FP64.
//
// Exact slices of B bits (B = 10 in the adjoint, 11 in the solve).  Each row
// of A, scaled by a power of two s (one s for all of the square part's rows,
// one per appended row) so that its largest entry is at most 2^(B-1) in
// magnitude, is written as a_1 + a_2 2^-B + a_3 2^-2B + ..., every a_k an
// integer in [-2^(B-1), 2^(B-1)] (exact in FP16).  The square part keeps three
// 10-bit slices in the adjoint (30 bits) and four 11-bit slices in the solve
// (44 bits), the appended rows six: their dot products with a centred x' can
// cancel, and three slices left ~1e-7 relative error in the gradient where six
// leave ~4e-9 (a CPU emulation of this scheme at n = 300..3000).  A slice times
// the integer dosages, accumulated by the tensor cores in FP32, is exact while
// every partial sum stays at most 2^24 in magnitude: one TMEM partial takes at
// most 2^24 / (2^(B-1) max|x'| 32) sub-chunks of 32 K (dosages, |x'| <= 2:
// 512 sub-chunks of 10-bit slices, 256 of 11-bit ones; any int8 values: at
// least two), and the epilogue adds the partials as int32.  The products leave as
// int32 and are combined per SNP in FP64 and int64, so the only error left is
// the slices' representation.
//
// Layout: A holds `slabs` slabs of RS rows (RS = 256 ceil((P + 1) / 2)), slab
// k = slice k of the square part's n_pad rows, then (slabs 0..2) slice k of
// the ne appended rows and their slice k + 3, then zero rows; FP16, row-major
// (K contiguous).  The product C = A x' is slabs RS x ncols int32,
// column-major (leading dimension slabs RS).
#include <cuda.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "gwas_internal.cuh"
#include "tc_ptx.cuh"
#include "trsm_tc_kernels.cuh"

namespace gwas {

using tc::EPI_COLS;
using tc::EPI_WARPS;
using tc::THREADS;
using tc::TN;
using tc::TRING;

namespace ex3 {
constexpr int KCH = 32;                              // FP16 K per sub-chunk: one 64-byte swizzle row
constexpr int SUB = 4;                               // sub-chunks per stage (128 K a stage, eight MMAs)
constexpr int KMMA = 16;                             // K per tcgen05.mma (kind::f16)
constexpr int CPB = TB / (KCH * SUB);                // stages per 128-wide K-block
constexpr int A_BYTES = TB * 64;                     // this CTA's 128 rows of a slice, one sub-chunk: 8 KB
constexpr int B_BYTES = (TN / 2) * 64;               // this CTA's 128 SNP columns, one sub-chunk: 8 KB
constexpr int STAGE_BYTES = SUB * (A_BYTES + B_BYTES);  // 64 KB: [A_0 .. A_3 | B_0 .. B_3]
// Three stages of eight MMAs: the single issuing thread waits on a stage and
// commits it once per eight MMAs (six stages of four ran 7 % slower).
constexpr int STAGES = 3;
constexpr int CHUNK_BYTES = 2048;                    // epilogue store chunk: 32 rows x 16 int32
constexpr int ST_COLS = 16;
constexpr int STG_OFF = STAGES * STAGE_BYTES;
constexpr int BAR_OFF = STG_OFF + EPI_WARPS * 2 * CHUNK_BYTES;
constexpr int NBARS = 2 * STAGES + 4 + 3 * TRING + 1;
constexpr int SMEM = 1024 + BAR_OFF + NBARS * 8 + TRING * 4 + 16;
static_assert(SMEM <= 232448, "shared memory per CTA");
constexpr int SLABS = 3;       // the adjoint: three 10-bit slices of W (30 bits)
constexpr int ADJ_BITS = 10;
constexpr int SOLVE_SLABS = SLICED_SLABS;  // the sliced solve: four 11-bit slices of W's triangle (44 bits)
constexpr int SOLVE_BITS = SLICED_BITS;

struct Params {
  CUtensorMap A;  // the stacked slices: dims {n_pad, slabs RS}, box {32, 128}, 64-byte swizzle, FP16
  CUtensorMap B;  // x' (FP16): dims {n_pad, bs}, box {32, 128}, 64-byte swizzle
  CUtensorMap C;  // the int32 product: dims {slabs RS, bs}, box {32, 16}
  int P;          // K-blocks of 128 (n_pad / 128)
  int U;          // row-panel pairs per slab (RS / 256)
  int RS;         // rows per slab
  int slabs;      // slices of the square part (3: the adjoint's W; 4: the solve's triangle)
  int amax;       // bound on |slice entry|: 2^(B-1) for B-bit slices (512 or 1024)
  int tri;        // 1: the square part is lower triangular (rows < 256 (u + 1) of pair u need
                  // K-blocks < 2u + 2 only) and units go out longest first
  int Cs;         // 256-column strips of the block
  int ncols;      // SNP columns of the block (the last strip may be partial)
  int ntiles;     // work units: slabs * U * Cs
  const int* xmax;         // largest |x'| of the block (set by the cast)
  unsigned int* counter;   // unit counter (zeroed by the cast)
  DevStatus* st;
  // the sliced solve (tri) only, else null: the epilogue of every pair wholly
  // inside the triangle forms sum_r x'_r (T_k x')_r over its rows and adds it to
  // acc[k * ldacc + column] (int64, exact: integer additions in any order) instead
  // of storing its rows of C; x' read from xc (FP16, leading dimension ldx)
  long long* acc;
  int ldacc;
  const __half* xc;
  int ldx;
};

// Sub-chunks (32 K each) per TMEM partial so that every partial sum is an
// integer of magnitude at most 2^24: amax * xmax * 32 * G <= 2^24 (G >= 2 for
// every int8 block: |x'| <= 255 and amax <= 1024).  `chunks`: a unit's most.
// A partial may end inside an operand stage.
__device__ __forceinline__ int partial_chunks(int xmax, int amax, int chunks) {
  if (xmax <= 0) return chunks;
  const long long g = (1LL << 24) / ((long long)amax * xmax * KCH);
  return g < 1 ? 1 : (g > chunks ? chunks : (int)g);
}

// The int32 totals hold amax * xmax * n_pad at most: beyond 2^31 the block is refused.
__device__ __forceinline__ bool in_range(int xmax, int amax, int P) {
  return (long long)amax * xmax * (long long)TB * P < (1LL << 31);
}

// Work unit t -> (slab, row-panel pair u, 256-column strip c) and its K-blocks.
// Dense: slab by slab.  Triangular: pair rows from the longest (all K-blocks)
// to the shortest over every slab and strip, so the launch ends on short units.
struct Unit {
  int slab, u, c, kend;
};
__device__ __forceinline__ Unit unit_of(const Params& b, int t) {
  Unit v;
  if (b.tri) {
    const int per = b.slabs * b.Cs;
    v.u = b.U - 1 - t / per;
    const int rem = t - (b.U - 1 - v.u) * per;
    v.slab = rem / b.Cs;
    v.c = rem - v.slab * b.Cs;
    v.kend = 2 * v.u + 2 <= b.P ? 2 * v.u + 2 : b.P;  // a pair of the triangle, or one holding appended rows
  } else {
    const int per = b.U * b.Cs;
    v.slab = t / per;
    const int rem = t - v.slab * per;
    v.u = rem / b.Cs;
    v.c = rem - v.u * b.Cs;
    v.kend = b.P;
  }
  return v;
}

__global__ void __launch_bounds__(THREADS, 1) exact_product_kernel(const __grid_constant__ Params b) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + BAR_OFF);
  uint64_t* full = bars;                 // CTA 0: both CTAs' loads of a stage
  uint64_t* empty = full + STAGES;       // CTA 0's commit: the stage's MMAs are done
  uint64_t* part_full = empty + STAGES;  // CTA 0's commit: a partial is complete
  uint64_t* part_empty = part_full + 2;  // CTA 0: both CTAs' epilogues are done with a partial
  uint64_t* tile_full = part_empty + 2;
  uint64_t* tile_empty = tile_full + TRING;
  uint64_t* peer_free = tile_empty + TRING;
  uint64_t* drain = peer_free + TRING;
  int* tile_ring = reinterpret_cast<int*>(drain + 1);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tile_ring + TRING);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
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
  const int xmax = *b.xmax;  // written by the cast, an ordinary launch before this one
  const bool ok_range = in_range(xmax, b.amax, b.P);
  if (!ok_range && blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(&st->err, DEV_OK, DEV_ERR_RANGE);
  const int ntiles = ok_range ? b.ntiles : 0;
  const int G = partial_chunks(xmax, b.amax, b.P * CPB * SUB);  // sub-chunks per TMEM partial

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
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
    ptx::prefetch_tensormap(&b.A);
    ptx::prefetch_tensormap(&b.B);
    ptx::prefetch_tensormap(&b.C);
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
          t = (ptx::aborting(st) || ntiles == 0) ? ntiles : (int)atomicAdd(b.counter, 1u);
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
        const Unit un = unit_of(b, t);
        const int arow = un.slab * b.RS + (2 * un.u + (int)rank) * TB;  // this CTA's 128 rows of A
        const int ycol = un.c * TN + (int)rank * (TN / 2);              // this CTA's 128 SNP columns
        bool ok = true;
        for (int j = 0; j < un.kend && ok; ++j) {
          for (int h = 0; h < CPB; ++h, ++cnt) {
            const int s = cnt % STAGES;
            const uint32_t r = cnt / STAGES;
            if (!ptx::mbar_wait(&empty[s], (r & 1) ^ 1, st)) { ok = false; break; }
            uint8_t* sb = smem + s * STAGE_BYTES;
            const int kx = j * TB + h * KCH * SUB;
            const uint32_t fb = lead_addr(&full[s]);
            if (leader)
              ptx::mbar_arrive_expect_tx(&full[s], 2 * STAGE_BYTES);
            else
              ptx::mbar_arrive_peer_count(fb);
#pragma unroll
            for (int u2 = 0; u2 < SUB; ++u2) {
              ptx::tma_load_2d_pair(sb + u2 * A_BYTES, &b.A, fb, kx + u2 * KCH, arow);
              ptx::tma_load_2d_pair(sb + SUB * A_BYTES + u2 * B_BYTES, &b.B, fb, kx + u2 * KCH, ycol);
            }
          }
        }
        if (!ok) break;
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------- MMA issuer (CTA 0 only)
    if (lane == 0) {
      constexpr uint32_t idesc = ptx::idesc_f32acc_f16(2 * TB, TN);
      uint32_t cnt = 0, kb = 0;
      for (int it = 0;; ++it) {
        const int slot = it % TRING;
        const uint32_t use = it / TRING;
        if (!ptx::mbar_wait_s<true>(&tile_full[slot], use & 1, st)) break;
        const int t = tile_ring[slot];
        ptx::mbar_arrive(&tile_empty[slot]);
        if (t >= ntiles) break;
        if (!leader) continue;
        const int nst = unit_of(b, t).kend * CPB;  // the unit's operand stages
        bool ok = true;
        int a = 0, left = 0;  // sub-chunks left for the current partial (a counter: no division)
        uint32_t d = 0, accumulate = 0;
        for (int g = 0; g < nst && ok; ++g, ++cnt) {
          const int s = cnt % STAGES;
          const uint32_t r = cnt / STAGES;
          if (!ptx::mbar_wait(&full[s], r & 1, st)) { ok = false; break; }
          ptx::tc_fence_after();
          const uint32_t base = ptx::smem_u32(smem + s * STAGE_BYTES);
#pragma unroll
          for (int u2 = 0; u2 < SUB; ++u2) {
            if (left == 0) {  // a fresh partial every G sub-chunks, alternating between the two buffers
              a = kb & 1;
              if (!ptx::mbar_wait(&part_empty[a], ((kb >> 1) & 1) ^ 1, st)) { ok = false; break; }
              ++kb;
              ptx::tc_fence_after();
              d = tmem_base + a * TN;
              accumulate = 0;
              left = G;
            }
#pragma unroll
            for (int kk = 0; kk < KCH / KMMA; ++kk) {
              const uint32_t off = kk * KMMA * 2;
              ptx::mma_pair<false>(d, ptx::sdesc_k64(base + u2 * A_BYTES + off),
                                   ptx::sdesc_k64(base + SUB * A_BYTES + u2 * B_BYTES + off), idesc, accumulate);
              accumulate = 1;
            }
            if (--left == 0) ptx::mma_commit_pair(&part_full[a], BOTH);
          }
          if (ok) ptx::mma_commit_pair(&empty[s], BOTH);
        }
        if (!ok) break;
        if (left != 0) ptx::mma_commit_pair(&part_full[a], BOTH);  // the unit's last partial
      }
    }
  } else if (warp >= 4) {
    // ----------------------------------------------------------------- epilogue
    constexpr int NT = 32 * EPI_WARPS;
    const int e = warp - 4;
    const int lq = e & 3;     // TMEM lanes (rows) 32 lq ..
    const int chalf = e >> 2;  // SNP columns chalf * 128 ..
    uint8_t* stg = smem + STG_OFF + e * 2 * CHUNK_BYTES;
    uint32_t kb = 0, gq = 0;
    int master[EPI_COLS];
    for (int it = 0;; ++it) {
      const int slot = it % TRING;
      const uint32_t use = it / TRING;
      if (!ptx::group_and(1, NT, ptx::mbar_wait_s<true>(&tile_full[slot], use & 1, st))) break;
      const int t = tile_ring[slot];
      ptx::named_bar(1, NT);
      if (lane == 0) ptx::mbar_arrive(&tile_empty[slot]);
      if (t >= ntiles) break;
      const Unit un = unit_of(b, t);
      const int nparts = (un.kend * CPB * SUB + G - 1) / G;
#pragma unroll
      for (int i = 0; i < EPI_COLS; ++i) master[i] = 0;
      bool ok = true;
      for (int pp = 0; pp < nparts && ok; ++pp) {
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
          for (int i = 0; i < 16; ++i) master[ch * 16 + i] += __float2int_rn(__uint_as_float(v[i]));  // exact
        }
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) count_lead(&part_empty[a]);
        ++kb;
      }
      if (!ok) break;
      if (b.acc != nullptr && 2 * un.u + 2 <= b.P) {
        // x'^T (T_k x') over this warp's 32 rows, column by column: the int64
        // product of each lane split at bit 20 (|x' C| < 2^39, so both parts sum
        // over 32 lanes inside an int32), one warp reduction each, one atomic
        // add per column.  Columns past the block's ncols (a partial last
        // strip) are neither read nor added: x' and acc hold the block's
        // columns only.
        const int rr = (2 * un.u + (int)rank) * TB + 32 * lq + lane;  // the row of T: x' row too
        const int cb = un.c * TN + chalf * EPI_COLS;
        const int nv = b.ncols - cb;  // valid columns of this warp's 128 (may be <= 0)
        const __half* xr = b.xc + rr;
        unsigned long long* ac = reinterpret_cast<unsigned long long*>(b.acc) + (size_t)un.slab * b.ldacc + cb;
#pragma unroll
        for (int q = 0; q < EPI_COLS / 8; ++q) {
          if (q * 8 >= nv) break;  // uniform over the warp
          int xv[8];
#pragma unroll
          for (int i = 0; i < 8; ++i)
            xv[i] = q * 8 + i < nv ? __half2int_rn(xr[(size_t)(cb + q * 8 + i) * b.ldx]) : 0;
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const long long pr = (long long)xv[i] * master[q * 8 + i];
            const unsigned lo = __reduce_add_sync(0xffffffffu, (unsigned)(pr & 0xFFFFF));
            const int hi = __reduce_add_sync(0xffffffffu, (int)(pr >> 20));
            if (lane == ((q * 8 + i) & 31) && q * 8 + i < nv)
              atomicAdd(ac + q * 8 + i, (unsigned long long)(((long long)hi << 20) + (long long)lo));
          }
        }
        continue;
      }
      // the tile's int32 products to HBM through TMA stores of 2 KB chunks
      const int r0 = un.slab * b.RS + (2 * un.u + (int)rank) * TB + 32 * lq;
      const int c0 = un.c * TN + chalf * EPI_COLS;
#pragma unroll
      for (int q = 0; q < EPI_COLS / ST_COLS; ++q) {
        uint8_t* buf = stg + (gq & 1) * CHUNK_BYTES;
        if (gq >= 2) {
          if (lane == 0) ptx::bulk_wait_read<1>();
          __syncwarp();
        }
        ++gq;
#pragma unroll
        for (int i = 0; i < ST_COLS; ++i) reinterpret_cast<int*>(buf)[i * 32 + lane] = master[q * ST_COLS + i];
        ptx::fence_proxy_async_shared();
        __syncwarp();
        if (lane == 0) {
          ptx::tma_store_2d(&b.C, buf, r0, c0 + q * ST_COLS);
          ptx::bulk_commit();
        }
      }
    }
    if (lane == 0) ptx::bulk_wait_all();  // the last stores have read the staging buffers
  }

  // ---------------------------------------------------------------- teardown
  if (warp == 1 && lane == 0 && leader) {
    ptx::mma_commit_pair(drain, 1);  // every MMA of the pair has completed before TMEM is released
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
}  // namespace ex3

// ----------------------------------------------------------- set-up kernels
// Largest |value| of each column of a column-major rows x ncols matrix (as the
// bits of a non-negative double, whose order is the integers').
__global__ void col_absmax_kernel(const double* __restrict__ X, int64_t ld, int rows, int ncols,
                                  unsigned long long* __restrict__ out) {
  const int col = blockIdx.y;
  if (col >= ncols) return;
  double m = 0.0;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x)
    m = fmax(m, fabs(X[r + (int64_t)col * ld]));
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out + col, (unsigned long long)__double_as_longlong(m));
}

// Slice k (0-based) of v s: a_0 = rint(v s), a_k = rint(2^B (remainder after
// a_0 .. a_{k-1})), step = 2^B.  Every step is exact in FP64 (a power-of-two
// scale, an integer subtracted); |remainder| <= 1/2, so |a_k| <= 2^(B-1).
__device__ __forceinline__ double slice_of(double v, double s, int k, double step) {
  double r = v * s, a = rint(r);
  for (int i = 0; i < k; ++i) {
    r = (r - a) * step;
    a = rint(r);
  }
  return a;
}

// The stacked slices A (slabs of RS rows, row-major, n_pad columns, FP16).
// Row R of slab k: R < n_pad: row R of the square part, W itself or (tri)
// its lower triangle with the diagonal halved, T (x'^T W x' = 2 x'^T T x');
// W is symmetric, so its row R is read as its column and the threads of a
// block read consecutive entries.  n_pad <= R < n_pad + 2 ne: appended row
// e = (R - n_pad) % ne (the columns of Ex, n_pad x ne), slice k for the first
// ne rows, slice k + 3 for the next, in slabs 0..2 (zero in later slabs).
// Further rows zero.
__global__ void slice_rows_kernel(const double* __restrict__ W, const double* __restrict__ Ex, int n_pad, int ne,
                                  int RS, int slabs, int tri, double step, const double* __restrict__ scale,
                                  __half* __restrict__ A) {
  const int R = blockIdx.y;
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= n_pad) return;
  double v = 0.0, s = 1.0;
  int k0 = 0, kind = 0;  // 1: square part, 2: appended row
  if (R < n_pad) {
    v = W[col + (int64_t)R * n_pad];
    if (tri) v = col < R ? v : (col == R ? 0.5 * v : 0.0);  // halving is exact
    s = scale[0];
    kind = 1;
  } else if (R < n_pad + 2 * ne) {
    const int e = (R - n_pad) % ne;
    k0 = (R - n_pad) / ne * 3;
    v = Ex[col + (int64_t)e * n_pad];
    s = scale[1 + e];
    kind = 2;
  }
  for (int k = 0; k < slabs; ++k) {
    const double a =
        kind == 1 ? slice_of(v, s, k, step) : (kind == 2 && k < 3) ? slice_of(v, s, k0 + k, step) : 0.0;
    A[((int64_t)k * RS + R) * n_pad + col] = __float2half_rn((float)a);  // an integer in [-1024, 1024]: exact
  }
}

// x' = x - c (c the SNP's integer shift, 0 without intercept) as FP16 on rows
// < n, 0 on rows n .. n_pad - 1; c stored in shift[col]; the largest |x'| of
// the block into *xmax.  One warp per SNP column; the block's first thread
// also zeroes the product's unit counter; acc (if not null): the fused sums
// of the sliced solve, slabs x ldacc, zeroed for the block's columns.
__global__ void cast_exact_kernel(const int8_t* __restrict__ X, int64_t ldx, int n, int n_pad, int ncols, int center,
                                  int8_t* __restrict__ shift, __half* __restrict__ xc, int* __restrict__ xmax,
                                  unsigned int* __restrict__ counter, long long* __restrict__ acc, int ldacc,
                                  int slabs) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *counter = 0;
  const int lane = threadIdx.x & 31;
  const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (col >= ncols) return;
  if (acc && lane < slabs) acc[(int64_t)lane * ldacc + col] = 0;
  const int8_t* x = X + (int64_t)col * ldx;
  int c = 0;
  if (center) {
    int sum = 0;
    for (int r = lane; r < n; r += 32) sum += x[r];
    for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    const long long num = 2LL * sum + n, den = 2LL * n;  // round half up of sum / n
    long long cc = num >= 0 ? num / den : -((-num + den - 1) / den);
    c = (int)(cc > 127 ? 127 : (cc < -127 ? -127 : cc));
  }
  if (lane == 0) shift[col] = (int8_t)c;
  int m = 0;
  __half* o = xc + (int64_t)col * n_pad;
  if ((reinterpret_cast<uintptr_t>(x) & 15) == 0) {  // 16 values a lane per step (n_pad: a multiple of 128)
    for (int r = lane * 16; r < n_pad; r += 32 * 16) {
      int8_t v8[16];
      if (r + 16 <= n) {
        *reinterpret_cast<int4*>(v8) = __ldg(reinterpret_cast<const int4*>(x + r));
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) v8[i] = r + i < n ? x[r + i] : 0;
      }
      __half2 h[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int a = r + 2 * i < n ? (int)v8[2 * i] - c : 0, b2 = r + 2 * i + 1 < n ? (int)v8[2 * i + 1] - c : 0;
        m = max(m, max(abs(a), abs(b2)));
        h[i] = __halves2half2(__int2half_rn(a), __int2half_rn(b2));
      }
      *reinterpret_cast<int4*>(o + r) = *reinterpret_cast<const int4*>(h);
      *reinterpret_cast<int4*>(o + r + 8) = *reinterpret_cast<const int4*>(h + 4);
    }
  } else {
    for (int r = lane; r < n_pad; r += 32) {
      const int v = r < n ? (int)x[r] - c : 0;
      m = max(m, abs(v));
      o[r] = __int2half_rn(v);
    }
  }
  for (int k = 16; k; k >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, k));
  if (lane == 0) atomicMax(xmax, m);
}

// y-gradient, first half: part[k][r] = sum over SNP chunk k of wp_i x'_ri,
// wp_i = wv[i p + p - 1] (the weight of the SNP column in W a_i), in
// double-FP32: wp_i = h_i + l_i (FP32 pieces), x' h_i exactly as the pair
// (p, fma(x', h_i, -p)) and the running sum as (s, c) with TwoSum steps --
// about 2^-44 relative, on the FP32 pipes instead of B300's narrow FP64 one.
constexpr int EX_DY_CHUNK = 128;
__global__ void __launch_bounds__(256) exact_dy_part_kernel(const __half* __restrict__ xc, int64_t ldc,
                                                            const double* __restrict__ wv, int p, int n, int ncols,
                                                            double* __restrict__ part) {
  __shared__ float wh[EX_DY_CHUNK], wl[EX_DY_CHUNK];
  const int i0 = blockIdx.y * EX_DY_CHUNK, i1 = min(i0 + EX_DY_CHUNK, ncols);
  for (int i = threadIdx.x; i < i1 - i0; i += blockDim.x) {
    const double w = wv[(int64_t)(i0 + i) * p + p - 1];
    const float h = (float)w;
    wh[i] = h;
    wl[i] = (float)(w - (double)h);
  }
  __syncthreads();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const __half* x = xc + r + (int64_t)i0 * ldc;
  float sh = 0.f, sl = 0.f;
#pragma unroll 4
  for (int i = 0; i < i1 - i0; ++i) {
    const float xv = __half2float(x[(int64_t)i * ldc]);
    const float pr = xv * wh[i];
    const float pe = fmaf(xv, wh[i], -pr);  // exact error of the product
    const float t = sh + pr;                // TwoSum(sh, pr)
    const float bv = t - sh;
    const float err = (sh - (t - bv)) + (pr - bv);
    sh = t;
    sl += err + pe + xv * wl[i];
  }
  part[(int64_t)blockIdx.y * n + r] = (double)sh + (double)sl;
}

// z = the chunk sums in order (rows < n; rows n .. n_pad - 1 zero)
__global__ void exact_dy_z_kernel(const double* __restrict__ part, int nchunks, int n, int n_pad,
                                  double* __restrict__ z) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_pad) return;
  double s = 0.0;
  if (r < n)
    for (int k = 0; k < nchunks; ++k) s += part[(int64_t)k * n + r];
  z[r] = s;
}

// dy[r] += sum_c W[r, c] z[c] + sum_a uT[a] X^_L[r, a]   (one warp per row,
// W symmetric: its row r is its column; 16-byte loads, four running sums)
__global__ void __launch_bounds__(256) exact_dy_apply_kernel(const double* __restrict__ W, int n_pad, int n,
                                                             const double* __restrict__ z,
                                                             const double* __restrict__ What,
                                                             const double* __restrict__ uT, int q,
                                                             double* __restrict__ dy) {
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= n) return;
  const double2* w = reinterpret_cast<const double2*>(W + (int64_t)r * n_pad);  // n_pad even, rows 16-byte aligned
  const double2* zz = reinterpret_cast<const double2*>(z);
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  const int n2 = n_pad / 2;  // z is zero past n
  int c = lane;
  for (; c + 96 < n2; c += 128) {  // four 16-byte loads in flight per lane
    double2 a[4], b[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) a[k] = __ldcs(w + c + 32 * k);
#pragma unroll
    for (int k = 0; k < 4; ++k) b[k] = zz[c + 32 * k];
    s0 = fma(a[0].x, b[0].x, s0);
    s1 = fma(a[0].y, b[0].y, s1);
    s2 = fma(a[1].x, b[1].x, s2);
    s3 = fma(a[1].y, b[1].y, s3);
    s0 = fma(a[2].x, b[2].x, s0);
    s1 = fma(a[2].y, b[2].y, s1);
    s2 = fma(a[3].x, b[3].x, s2);
    s3 = fma(a[3].y, b[3].y, s3);
  }
  for (; c < n2; c += 32) {
    const double2 a = __ldcs(w + c), za = zz[c];
    s0 = fma(a.x, za.x, s0);
    s1 = fma(a.y, za.y, s1);
  }
  double s = (s0 + s1) + (s2 + s3);
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    for (int a = 0; a < q; ++a) s = fma(uT[a], What[r + (int64_t)a * n_pad], s);
    dy[r] += s;
  }
}

// ------------------------------------------------------------------- host side
// One state serves both uses of the exact products: the adjoint (W dense in 3
// slabs; appended rows [X^_L | y^ | W X^_L | W y^]) and the sliced solve (W's
// triangle T in 4 slabs; appended rows [X^_L | Y^]).
struct ExactProducts {
  int n = 0, n_pad = 0, q = 0, bs = 0, P = 0, U = 0, RS = 0, ne = 0, slabs = 0;
  int bits = 0;  // bits per slice
  bool tri = false, center = false;
  int max_clusters = 0;
  double* W = nullptr;          // n_pad x n_pad FP64 (owned; kept by the adjoint for its y-gradient)
  __half* A = nullptr;          // slabs RS x n_pad FP16 slices
  __half* xc = nullptr;         // n_pad x bs FP16 x'
  int32_t* C = nullptr;         // slabs RS x bs int32 products
  int8_t* shift = nullptr;      // bs
  int* xmax = nullptr;          // [0] largest |x'|; [1..] the unit counter
  double* inv_scale = nullptr;  // [0] 1 / s_W, [1 + e] 1 / s_e
  double* part = nullptr;       // the adjoint's y-gradient chunk partials
  double* z = nullptr;          // n_pad (adjoint)
  long long* acc = nullptr;     // the sliced solve's fused sums: slabs x bs int64
  ex3::Params prm;
};

void exact_destroy(ExactProducts* E) {
  if (!E) return;
  cudaFree(E->W);
  cudaFree(E->A);
  cudaFree(E->xc);
  cudaFree(E->C);
  cudaFree(E->shift);
  cudaFree(E->xmax);
  cudaFree(E->inv_scale);
  cudaFree(E->part);
  cudaFree(E->z);
  cudaFree(E->acc);
  delete E;
}

// 2^e with mx 2^e <= bound < mx 2^(e+1); 1 for a zero row
static double pow2_scale(double mx, double bound) {
  if (!(mx > 0.0) || !std::isfinite(mx)) return 1.0;
  int e = (int)std::floor(std::log2(bound / mx));
  while (std::ldexp(mx, e) > bound) --e;
  while (std::ldexp(mx, e + 1) <= bound) ++e;
  return std::ldexp(1.0, e);
}

// W (taken over), Ex = the ne appended columns (n_pad x ne, read here only).
static cudaError_t exact_create(ExactProducts** out, double* W, const double* Ex, int ne, int slabs, int bits,
                                bool tri, bool keep_w, int n, int n_pad, int q, int bs, bool center, int num_sms,
                                cudaStream_t s, int64_t* launches) {
  *out = nullptr;
  ExactProducts* E = new ExactProducts;
  E->W = W;
  E->n = n;
  E->n_pad = n_pad;
  E->q = q;
  E->bs = bs;
  E->P = n_pad / TB;
  E->U = (E->P + 2) / 2;  // row-panel pairs over W's P panels and one panel of appended rows
  E->RS = 2 * E->U * TB;
  E->ne = ne;
  E->slabs = slabs;
  E->bits = bits;
  E->tri = tri;
  E->center = center;
  cudaError_t e;
#define TRY(x)            \
  do {                    \
    e = (x);              \
    if (e != cudaSuccess) { \
      exact_destroy(E);   \
      return e;           \
    }                     \
  } while (0)
  const size_t rows = (size_t)slabs * E->RS;
  TRY(cudaMalloc(&E->A, sizeof(__half) * rows * n_pad));
  TRY(cudaMalloc(&E->xc, sizeof(__half) * (size_t)n_pad * bs));
  TRY(cudaMalloc(&E->C, sizeof(int32_t) * rows * bs));
  TRY(cudaMalloc(&E->shift, (size_t)bs));
  TRY(cudaMalloc(&E->xmax, 64));
  TRY(cudaMalloc(&E->inv_scale, sizeof(double) * (1 + ne)));
  if (tri) TRY(cudaMalloc(&E->acc, sizeof(long long) * (size_t)slabs * bs));
  if (keep_w) {
    const int nchunks = (bs + EX_DY_CHUNK - 1) / EX_DY_CHUNK;
    TRY(cudaMalloc(&E->part, sizeof(double) * (size_t)nchunks * n));
    TRY(cudaMalloc(&E->z, sizeof(double) * (size_t)n_pad));
  }
  TRY(cudaMemsetAsync(E->xc, 0, sizeof(__half) * (size_t)n_pad * bs, s));
  // scales: the largest entry of W (bounds T's too) and of every appended row
  unsigned long long* mx = nullptr;
  TRY(cudaMallocAsync(&mx, sizeof(unsigned long long) * (size_t)(n_pad + ne), s));
  TRY(cudaMemsetAsync(mx, 0, sizeof(unsigned long long) * (size_t)(n_pad + ne), s));
  col_absmax_kernel<<<dim3(8, n_pad), 256, 0, s>>>(W, n_pad, n_pad, n_pad, mx);
  col_absmax_kernel<<<dim3(8, ne), 256, 0, s>>>(Ex, n_pad, n_pad, ne, mx + n_pad);
  *launches += 2;
  TRY(cudaGetLastError());
  std::vector<unsigned long long> hm((size_t)n_pad + ne);
  TRY(cudaMemcpyAsync(hm.data(), mx, sizeof(unsigned long long) * hm.size(), cudaMemcpyDeviceToHost, s));
  TRY(cudaStreamSynchronize(s));
  double wmax = 0.0;
  for (int i = 0; i < n_pad; ++i) {
    double v;
    std::memcpy(&v, &hm[i], sizeof v);
    wmax = std::max(wmax, v);
  }
  std::vector<double> sc(1 + ne), inv(1 + ne);
  const double amax = std::ldexp(1.0, bits - 1);  // the largest |slice entry|
  sc[0] = pow2_scale(wmax, amax);
  for (int i = 0; i < ne; ++i) {
    double v;
    std::memcpy(&v, &hm[(size_t)n_pad + i], sizeof v);
    sc[1 + i] = pow2_scale(v, amax);
  }
  for (int i = 0; i <= ne; ++i) inv[i] = 1.0 / sc[i];  // powers of two: exact
  double* dsc = nullptr;
  TRY(cudaMallocAsync(&dsc, sizeof(double) * (1 + ne), s));
  TRY(cudaMemcpyAsync(dsc, sc.data(), sizeof(double) * (1 + ne), cudaMemcpyHostToDevice, s));
  TRY(cudaMemcpyAsync(E->inv_scale, inv.data(), sizeof(double) * (1 + ne), cudaMemcpyHostToDevice, s));
  slice_rows_kernel<<<dim3((n_pad + 255) / 256, E->RS), 256, 0, s>>>(W, Ex, n_pad, ne, E->RS, slabs, tri ? 1 : 0,
                                                                     2.0 * amax, dsc, E->A);
  *launches += 1;
  TRY(cudaGetLastError());
  TRY(cudaFreeAsync(mx, s));
  TRY(cudaFreeAsync(dsc, s));
  TRY(cudaStreamSynchronize(s));
  if (!keep_w) {
    cudaFree(E->W);
    E->W = nullptr;
  }
  // tensor maps and the launch parameters (the block width fixed at bs; a
  // shorter block covers only its strips)
  tc::EncodeTiledFn enc = nullptr;
  TRY(tc::get_encode(&enc));
  ex3::Params& p = E->prm;
  std::memset(&p, 0, sizeof p);
  TRY(tc::make_map(enc, &p.A, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, E->A, n_pad, rows, 2 * (size_t)n_pad, ex3::KCH, TB,
                   true));
  TRY(tc::make_map(enc, &p.B, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, E->xc, n_pad, bs, 2 * (size_t)n_pad, ex3::KCH, TN / 2,
                   true));
  TRY(tc::make_map(enc, &p.C, CU_TENSOR_MAP_DATA_TYPE_INT32, E->C, rows, bs, 4 * rows, 32, ex3::ST_COLS, false));
  p.P = E->P;
  p.U = E->U;
  p.RS = E->RS;
  p.slabs = slabs;
  p.amax = 1 << (bits - 1);
  p.tri = tri ? 1 : 0;
  p.xmax = E->xmax;
  p.counter = reinterpret_cast<unsigned int*>(E->xmax + 1);
  p.acc = E->acc;
  p.ldacc = bs;
  p.xc = E->xc;
  p.ldx = n_pad;
  TRY(cudaFuncSetAttribute(ex3::exact_product_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, ex3::SMEM));
  {
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof cfg);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2 * (num_sms / 2));
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = ex3::SMEM;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    TRY(cudaOccupancyMaxActiveClusters(&E->max_clusters, ex3::exact_product_kernel, &cfg));
    if (E->max_clusters < 1) TRY(cudaErrorLaunchOutOfResources);
  }
#undef TRY
  *out = E;
  return cudaSuccess;
}

cudaError_t exact_adjoint_create(ExactProducts** out, double* W, const double* What, const double* W2, int n,
                                 int n_pad, int q, int bs, bool center, int num_sms, cudaStream_t s,
                                 int64_t* launches) {
  *out = nullptr;
  const int ne = 2 * (q + 1);
  double* Ex = nullptr;  // the appended columns [X^_L | y^ | W X^_L | W y^] side by side
  cudaError_t e = cudaMallocAsync(&Ex, sizeof(double) * (size_t)n_pad * ne, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(Ex, What, sizeof(double) * (size_t)n_pad * (q + 1), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(Ex + (size_t)n_pad * (q + 1), W2, sizeof(double) * (size_t)n_pad * (q + 1),
                        cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) {
    if (Ex) cudaFreeAsync(Ex, s);
    cudaFree(W);
    return e;
  }
  e = exact_create(out, W, Ex, ne, ex3::SLABS, ex3::ADJ_BITS, false, true, n, n_pad, q, bs, center, num_sms, s,
                   launches);
  cudaFreeAsync(Ex, s);
  return e;
}

cudaError_t exact_solve_create(ExactProducts** out, double* W, const double* Wh, int nw, int n, int n_pad, int q,
                               int bs, bool center, int num_sms, cudaStream_t s, int64_t* launches) {
  return exact_create(out, W, Wh, nw, ex3::SOLVE_SLABS, ex3::SOLVE_BITS, true, false, n, n_pad, q, bs, center,
                      num_sms, s, launches);
}

// x' of a block into the FP16 operand (columns past ncols of the last strip
// zeroed), then the product C = A x' over the block's strips.
static cudaError_t exact_cast_product(ExactProducts* E, const int8_t* X, int64_t ldx, int ncols, DevStatus* st,
                                      cudaStream_t s, cudaEvent_t k0, cudaEvent_t k1) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(E->xmax, 0, sizeof(int), s)) != cudaSuccess) return e;
  // the last strip's columns past ncols: zeros, not an earlier block's values
  const int cover = std::min(E->bs, (ncols + TN - 1) / TN * TN);
  if (cover > ncols &&
      (e = cudaMemsetAsync(E->xc + (size_t)ncols * E->n_pad, 0, sizeof(__half) * (size_t)(cover - ncols) * E->n_pad,
                           s)) != cudaSuccess)
    return e;
  cast_exact_kernel<<<(ncols + 7) / 8, 256, 0, s>>>(X, ldx, E->n, E->n_pad, ncols, E->center ? 1 : 0, E->shift,
                                                    E->xc, E->xmax, reinterpret_cast<unsigned int*>(E->xmax + 1),
                                                    E->acc, E->bs, E->slabs);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  ex3::Params p = E->prm;
  p.Cs = (ncols + TN - 1) / TN;
  p.ncols = ncols;
  p.ntiles = E->slabs * p.U * p.Cs;
  p.st = st;
  const int ncl = std::min(p.ntiles, E->max_clusters);
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof cfg);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(2 * ncl);
  cfg.blockDim = dim3(THREADS);
  cfg.dynamicSmemBytes = ex3::SMEM;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (k0 && (e = cudaEventRecord(k0, s)) != cudaSuccess) return e;
  if ((e = cudaLaunchKernelEx(&cfg, ex3::exact_product_kernel, p)) != cudaSuccess) return e;
  if (k1 && (e = cudaEventRecord(k1, s)) != cudaSuccess) return e;
  return cudaSuccess;
}

cudaError_t exact_adjoint_block(ExactProducts* E, const int8_t* X, int64_t ldx, int ncols, const SolveConsts* sc,
                                const double* GH, const double* What, double h, double sigma2, double* chi2,
                                double* dh, double* wv, double* uT, double* dh_accum, double* dy_accum,
                                DevStatus* st, cudaStream_t s, int64_t* launches) {
  if (ncols <= 0) return cudaSuccess;
  if (ncols > E->bs || E->tri || !E->W) return cudaErrorInvalidValue;
  cudaError_t e;
  if ((e = exact_cast_product(E, X, ldx, ncols, st, s, nullptr, nullptr)) != cudaSuccess) return e;
  const int64_t ldc = (int64_t)E->slabs * E->RS;
  if ((e = launch_exact_adjoint_sums(E->C, ldc, E->RS, E->xc, E->n_pad, E->n, E->n_pad, E->ne, E->inv_scale, sc, GH,
                                     E->q, ncols, h, sigma2, E->xmax, chi2, dh, wv, dh_accum, uT, s)) != cudaSuccess)
    return e;
  const int p1 = E->q + 1, nchunks = (ncols + EX_DY_CHUNK - 1) / EX_DY_CHUNK;
  exact_dy_part_kernel<<<dim3((E->n + 255) / 256, nchunks), 256, 0, s>>>(E->xc, E->n_pad, wv, p1, E->n, ncols,
                                                                         E->part);
  exact_dy_z_kernel<<<(E->n_pad + 255) / 256, 256, 0, s>>>(E->part, nchunks, E->n, E->n_pad, E->z);
  exact_dy_apply_kernel<<<(E->n + 7) / 8, 256, 0, s>>>(E->W, E->n_pad, E->n, E->z, What, uT, E->q, dy_accum);
  *launches += 7;
  return cudaGetLastError();
}

int exact_max_ctas(const ExactProducts* E) { return E ? 2 * E->max_clusters : 0; }

cudaError_t exact_solve_product(ExactProducts* E, const int8_t* X, int64_t ldx, int ncols, DevStatus* st,
                                cudaStream_t s, cudaEvent_t k0, cudaEvent_t k1) {
  if (ncols <= 0) return cudaSuccess;
  if (ncols > E->bs || !E->tri) return cudaErrorInvalidValue;
  return exact_cast_product(E, X, ldx, ncols, st, s, k0, k1);
}

cudaError_t exact_solve_sums(ExactProducts* E, int ncols, const SolveConsts* sc, int t, double* b, double* se,
                             int* status, cudaStream_t s) {
  if (ncols <= 0) return cudaSuccess;
  if (ncols > E->bs || !E->tri) return cudaErrorInvalidValue;
  // rows of T stored as products: those of the last row-panel pair (it also holds the appended rows)
  const int r_lo = 2 * (E->U - 1) * TB;
  return launch_sliced_solve(E->C, (int64_t)E->slabs * E->RS, E->RS, E->acc, E->bs, r_lo, E->xc, E->n_pad, E->n,
                             E->ne, E->inv_scale, sc, E->q, t, ncols, b, se, status, E->center ? E->shift : nullptr, s);
}

}  // namespace gwas
