// Split-precision blocked triangular solve on the sm_103a tensor cores.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "gwas_internal.cuh"

namespace gwas {
namespace tc {

enum Split : int { SPLIT_BF16 = 0, SPLIT_TF32 = 1 };

struct TcState;

// Splits the FP64 block operator Aop into hi + lo pieces (BF16 or TF32) and
// allocates the per-block buffers for up to bs SNP columns.
cudaError_t create(TcState** out, Split split, const double* Aop, int n, int n_pad, int bs, int num_sms,
                   DevStatus* st, cudaStream_t s, int64_t* launches);

// X~ = L^-1 X for ncols <= bs int8 columns (X 16-byte aligned, ldx % 16 == 0).
// The FP32 result is left in xt_f32() with leading dimension xt_ld().
cudaError_t run_block(TcState* t, const int8_t* X, int64_t ldx, int ncols, cudaStream_t s, int64_t* launches);

const float* xt_f32(const TcState* t);
int64_t xt_ld(const TcState* t);
void destroy(TcState* t);

}  // namespace tc
}  // namespace gwas
