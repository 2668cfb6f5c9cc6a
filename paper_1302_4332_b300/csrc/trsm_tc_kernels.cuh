// The split-precision solve's kernels (trsm_tc.cu) and their host side
// (trsm_tc_host.cu) share this: tile geometry, the launch parameter block
// (one or several studies' tensor maps and buffers) and the kernels' launch
// entry points.
#pragma once

#include <cuda.h>

#include <cstdint>

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
// one, the substitution's tile modes give the same results bit for bit.  (The
// inverse form puts the first two K-blocks of a unit into one partial.)
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
  const float* rscale;  // inverse form with FP16 pieces: row r of L^-1 was split scaled by 1 / rscale[r]
  // inverse form, per-SNP sums formed by the epilogue in place of storing X~
  // (red null: X~ is stored for a separate reduction pass): W = [X~_L | Y~] in
  // FP32, row-major, row stride ws (4 or 8), nw <= ws columns; the partial
  // sums for SNP column j, a < nw: x~ . W[:, a], a = nw: x~ . x~, over the 128
  // rows of row panel k at red[(k (nw + 1) + a) ldr + j] (ws 4), or over the
  // 32 rows of its quarter g at red[((4k + g)(nw + 1) + a) ldr + j] (ws 8)
  const float* w32;
  float* red;
  int ws, nw;
  int64_t ldr;
};

// The tensor maps of one study: block operator hi/lo, X~ hi/lo, int8 block.
struct TcMaps {
  CUtensorMap Ahi, Alo, Bhi, Blo, X8;
  CUtensorMap BhiH, BloH, X8H;  // half-width boxes (128 SNP columns) for the pair modes
  CUtensorMap StX, StHi, StLo;  // pair product's epilogue stores: FP32 X~, hi piece (BF16), lo piece
  CUtensorMap XcH;              // inverse form: the cast block x - c_i (BF16/FP32), half-width boxes
};

// A launch over one or several studies (the batching form): tiles of all
// studies are handed out from one counter in the order of `order`, which
// interleaves the studies row panel by row panel so that every study's
// dependency chain advances while the SMs stay busy.
struct TcBatch {
  TcMaps maps[MAX_STUDIES];
  TcStudy s0;                 // the study when there is only one (order == null)
  const TcStudy* studies;     // device copies of the studies when order != null (null: s0 alone)
  const uint32_t* order;      // tile t -> (study << 28) | (k << 14) | c
  int nstudies, ntiles;
  unsigned int* counter;
  DevStatus* st;
};

namespace pair2 {
// SNP columns per 2 KB epilogue store chunk of the pair product (32 rows):
// BF16 mode stores hi+lo chunks (4 B per element), then FP32 chunks; TF32
// mode FP32+lo chunks (8 B)
template <bool TF32>
constexpr int st_cols() { return TF32 ? 8 : 16; }
}  // namespace pair2

namespace inv2 {
constexpr int ST_COLS = 16;  // SNP columns per inverse-form store chunk (32 rows x 16 FP32 = 2 KB)
}  // namespace inv2

// cuTensorMapEncodeTiled through the runtime's driver entry point, and a 2D
// tiled map: dims {inner, outer}, outer stride in bytes, box {bi, bo};
// swz: the 64-byte swizzle of the operand stages (box inner extent 64 bytes).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
cudaError_t get_encode(EncodeTiledFn* fn);
cudaError_t make_map(EncodeTiledFn enc, CUtensorMap* m, CUtensorMapDataType dt, const void* base, uint64_t inner,
                     uint64_t outer, uint64_t stride_bytes, uint32_t bi, uint32_t bo, bool swz);

// Launch entry points of the kernels (trsm_tc.cu).
// Opt-in shared memory of the forward kernels (clusters: also the pair and
// inverse-form kernels).  f16: the inverse form's FP16 variant (TILES_INVERSE
// only, tf32 false).
cudaError_t set_kernel_attrs(bool tf32, bool clusters);
// Co-resident 2-CTA clusters of a cluster-mode kernel (one CTA per SM).
cudaError_t query_clusters(bool tf32, TileMode mode, int num_sms, int* out, bool f16 = false);
// One launch over b.ntiles work units (tiles, or row-panel pairs of a strip).
// stages: operand stages of the inverse-form kernel (8 or 6; other modes: 8).
cudaError_t launch_solve(bool tf32, TileMode mode, const TcBatch& b, int num_sms, int max_clusters,
                         cudaStream_t s, bool f16 = false, int stages = 8);

}  // namespace tc
}  // namespace gwas
