// Split-precision blocked triangular solve on the sm_103a tensor cores.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "gwas_internal.cuh"

namespace gwas {
namespace tc {

// SPLIT_F16: the inverse form only, L^-1 split into FP16 hi + lo after a
// power-of-two scaling of each row (the rest of such a context runs in BF16).
enum Split : int { SPLIT_BF16 = 0, SPLIT_TF32 = 1, SPLIT_F16 = 2 };

// How tiles (row panel k, strip c) map onto CTAs.
enum TileMode : int {
  TILES_AUTO = 0,            // the measured fastest for the split (resolved by create)
  TILES_SINGLE = 1,          // every tile on its own CTA
                             // (2 is not a mode)
  TILES_PAIR_MMA = 3,        // panels 2u, 2u+1: one M = 256 product on a 2-CTA cluster (cta_group::2)
  TILES_INVERSE = 4,         // L^-1 formed at set-up; a block is the triangular product L^-1 X, row-panel
                             // pairs as M = 256 products on 2-CTA clusters, no dependency between tiles
};

struct TcState;

// Splits the FP64 block operator Aop into hi + lo pieces (BF16 or TF32) and
// allocates the per-block buffers for up to bs SNP columns.  TILES_INVERSE
// instead forms L^-1 from Aop (the TF32x3 pair product on the identity,
// 4096 columns per launch) and splits that.  center: X_L's
// first column is the intercept, so every SNP column is solved shifted by the
// integer nearest its mean (exact in BF16/TF32; the reductions map the results
// back), which removes most of the cancellation between the SNP and the
// intercept in S_BR - S_BL S_TL^-1 S_BL^T.
// strip_group > 0: tiles go out row panel by row panel over groups of that
// many column strips (the strips' X~ stays in L2 while it is re-read).
cudaError_t create(TcState** out, Split split, const double* Aop, int n, int n_pad, int bs, int num_sms,
                   bool center, DevStatus* st, cudaStream_t s, int64_t* launches, int strip_group = 0,
                   TileMode mode = TILES_AUTO);

// X~ = L^-1 X for ncols <= bs int8 columns (X 16-byte aligned, ldx % 16 == 0).
// The FP32 result is left in xt_f32() with leading dimension xt_ld() (the
// inverse form with the sums in its epilogue leaves partials() instead).
// ev0 / ev1 (optional): recorded on s right before and after the solve kernel.
cudaError_t run_block(TcState* t, const int8_t* X, int64_t ldx, int ncols, cudaStream_t s, int64_t* launches,
                      cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr, bool packed = false);
// run_block takes 2-bit packed columns (packed = true, ldx >= ceil(n/4) bytes a
// column, 16-byte aligned): the inverse form at n <= 16384, whose cast reads them.
bool packed_ok(const TcState* t);

// The batching form: one persistent launch over several studies (each with its
// own operator and buffers; all BF16 or all TF32).  ts[i] solves ncols[i]
// columns of X[i]; results land in each study's xt_f32().
struct TcBatchState;
cudaError_t batch_create(TcBatchState** out, TcState* const* ts, int nstudies);
// Fixes the geometry of later launches (device blocks X[i], ncols[i];
// order_mode 0 interleaves the studies row panel by row panel, 1 runs them
// one after another); synchronizes the stream.
cudaError_t batch_plan(TcBatchState* B, TcState* const* ts, const int8_t* const* X, const int64_t* ldx,
                       const int* ncols, int order_mode, cudaStream_t s, int strip_group = 0);
// One launch of the planned batch (stream-ordered only: capturable).
cudaError_t batch_launch(TcBatchState* B, TcState* const* ts, cudaStream_t s, int64_t* launches);
// Operand stages of the inverse-form kernel in later launches: 8 (default) or 6.
cudaError_t batch_set_stages(TcBatchState* B, int stages);
void batch_destroy(TcBatchState* B);
constexpr int kMaxBatchStudies = 8;

const float* xt_f32(const TcState* t);
// Inverse form: the per-SNP sums of x~ with W = [X~_L | Y~] (FP32, row-major,
// row stride ws = 4 or 8, nw <= 8 columns) and of x~ with itself formed by the
// solve's epilogue, which then stores no X~.  Other modes or sizes: no change
// (the sums stay a separate pass over xt_f32()).
cudaError_t set_reductions(TcState* t, const float* w32, int ws, int nw);
// Precision studies (inverse form): zeroes the lo piece of L^-1, so that the
// solve multiplies by its hi piece alone.  Other modes: cudaErrorInvalidValue.
cudaError_t drop_lo_piece(TcState* t, cudaStream_t s);
// The last block's partial sums, or null when the block stored X~ instead:
// partial_groups(t) row groups x (nw + 1) quantities, each a plane of
// partial_ld(t) floats with SNP column j at offset j.
const float* partials(const TcState* t);
int partial_groups(const TcState* t);
int64_t partial_ld(const TcState* t);
const CUtensorMap* xt_reduce_map(const TcState* t);  // xt_f32() as the reduction's tiled map
const int8_t* shift_of(const TcState* t);  // per-SNP shifts of the last block, or null
int64_t xt_ld(const TcState* t);
TileMode tile_mode(const TcState* t);  // the resolved mode
// CTAs of a launch over a full block (bs columns) and its cluster size.
void launch_shape(const TcState* t, int* ctas, int* cluster_size);
void destroy(TcState* t);

}  // namespace tc
}  // namespace gwas
