// Internal declarations of the gwas_b300 CUDA library (sm_103a).
//
// Device layout of one study (n samples, n_pad = n rounded up to TB):
//   L     n_pad x n_pad FP64, column-major: the lower Cholesky factor of M
//         (Sec. 2.1 "potrf M"); padded rows/columns hold the identity.
//   Dinv  P = n_pad / TB diagonal-block inverses D_k^-1 = L_kk^-1, TB x TB each,
//         column-major, FP64.
//   Aop   n_pad x n_pad FP64, ROW-major: the block operator of the blocked
//         triangular solve.  Row panel k holds
//             [ -D_k^-1 L_k0 | ... | -D_k^-1 L_k,k-1 | D_k^-1 ]
//         so that X~_k = D_k^-1 X_k + sum_{j<k} (-D_k^-1 L_kj) X~_j is one
//         product per row panel (Sec. 2.2: the trsm over a block of SNPs).
//         Row-major = the reduction index is contiguous for every row.
//   W     n_pad x (q+1) FP64, column-major: [X~_L | y~] (Listing 1 precompute).
//   Xt    n_pad x bs: X~_b = L^-1 X_b for the current block of SNPs.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/gwas_b300.h"

namespace gwas {

constexpr int TB = 128;             // diagonal block (row panel) size of the blocked solve
constexpr int F64_TN = 64;          // SNP columns per tile of the FP64 solve
constexpr int QMAX = 15;            // most fixed covariates (p <= 16)
constexpr double SINGULAR_TAU = 1e-7;
constexpr long long WAIT_LIMIT_NS = 8000000000LL;  // bounded device-side waits: 8 s

// Codes the kernels write into DevStatus::err.
// DEV_ERR_RANGE: the split adjoint's exact products refused a block whose
// largest |x - c| times 512 n_pad reaches 2^31 (never for dosages 0..2).
enum : int { DEV_OK = 0, DEV_ERR_TIMEOUT = 1, DEV_ERR_RANGE = 2 };

// Device-resident status block of a context.
struct DevStatus {
  int err;                      // first device-side error (DEV_*)
  int abort;                    // set when a persistent kernel gives up; others drain
  unsigned long long not_spd;   // smallest failing Cholesky pivot, ~0ull if none
  int sc_err;                   // S_TL not positive definite
  int pad[3];
};

// Per-SNP solve constants from the loop-invariant part of Listing 1.
// With S_TL = C C^T:  Cinv = C^-1, zT = C^-1 r_T, b0 = S_TL^-1 r_T,
// dSTL_j = (S_TL^-1)_jj; zT and b0 per phenotype (t phenotypes share M, X_L and
// so S_TL; r_T = X~_L^T y~ differs).
constexpr int TMAX = 16;  // phenotypes sharing one study (q + t <= QMAX + 1 columns of W)
struct SolveConsts {
  int q;
  int t;
  double Cinv[QMAX * QMAX];  // column-major q x q (leading dimension QMAX)
  double zT[TMAX][QMAX];
  double b0[TMAX][QMAX];
  double dSTL[QMAX];
  double stl00;  // S_TL[0][0] (uncentered S_BR of a shifted SNP, see reduce_solve.cu)
};

// Scheduler state of one persistent triangular-solve launch.
struct Sched {
  unsigned int counter;  // next tile to hand out
  unsigned int pad[31];
  // followed by int flags[P * C]: tile (k, c) finished
};

__host__ __device__ inline int* sched_flags(Sched* s) { return reinterpret_cast<int*>(s + 1); }

// ---- launchers (each returns the cudaError_t of its launch) ----

// a1: A = sigma2 (h Phi + (1-h) I) on the lower triangle (or a copy of a given L),
// identity on the padding, zero strict upper triangle.
cudaError_t launch_form_m(const double* phi, int64_t ldphi, int n, int n_pad, double h, double sigma2,
                          int is_L, double* A, cudaStream_t s);

// a2 + a4: blocked right-looking Cholesky of A (n_pad x n_pad) in place; writes
// the diagonal-block inverses into Dinv.  panel is n_pad x TB scratch.
// Counts its launches into *launches.
cudaError_t launch_potrf(double* A, int n_pad, double* Dinv, double* panel, DevStatus* st, cudaStream_t s,
                         int64_t* launches);

// a4 for a caller-supplied L: checks its diagonal and inverts its diagonal blocks.
cudaError_t launch_invert_diag_blocks(double* L, int n_pad, double* Dinv, DevStatus* st, cudaStream_t s);

// a4: the block operator Aop (row-major) from L and Dinv.
cudaError_t launch_build_aop(const double* L, const double* Dinv, int n_pad, double* Aop, cudaStream_t s,
                             int64_t* launches);

// a6 (FP64): Xt = L^-1 X for ncols columns of X (TIn = int8_t or double).
struct TrsmF64Args {
  const double* Aop;
  int64_t lda;        // n_pad
  const void* X;      // input columns
  int64_t ldx;
  int n;              // valid rows of X (rows >= n read as 0)
  double* Xt;
  int64_t ldt;        // n_pad
  int P;              // row panels
  int ncols;
  int C;              // column tiles (of F64_TN)
  Sched* sched;
  DevStatus* st;
  // >= 0 (lower solve only): X holds identity columns tri_col0 .. tri_col0 + ncols - 1,
  // so rows above each column strip's first column are zero in X and X~: those
  // tiles are written as zeros without the solve and later tiles skip them
  int64_t tri_col0 = -1;
};
// upper = true: Xt = L^-T X with Aop the transpose block operator (FP64 input only).
cudaError_t launch_trsm_f64(const TrsmF64Args& a, bool int8_input, cudaStream_t s, int num_sms,
                            bool upper = false);
// CTAs of the FP64 solve when there are at least that many tiles.
int trsm_f64_grid(int num_sms);

// The transpose block operator (row-major): row panel k holds D_k^-T at
// block k and -D_k^-T L_jk^T at blocks j > k.
cudaError_t launch_build_aop_t(const double* L, const double* Dinv, int n_pad, double* AopT, cudaStream_t s,
                               int64_t* launches);

// a3: G = W^T W (nc x nc, column-major), W n_pad x nc.
cudaError_t launch_gram(const double* W, int64_t ldw, int n_pad, int nc, double* G, cudaStream_t s);
// a3: solve constants from G (q covariates), flags S_TL not SPD in st->sc_err.
cudaError_t launch_solve_consts(const double* G, int q, int t, SolveConsts* sc, DevStatus* st, cudaStream_t s);

// a7 + a8: per-SNP reductions against W and the p x p solve.
enum XtKind : int { XT_F64 = 0, XT_F32 = 1 };
// XT_F64 reads W (FP64, column-major, ldw); XT_F32 reads W32 (FP32, row-major,
// row stride w32_stride(q), made by launch_make_w32).  shift (XT_F32 only, may
// be null): per-SNP integer c_i the SNP column was shifted by before the solve
// (x' = x - c_i * X_L[:, 0], X_L[:, 0] the intercept); results are mapped back
// to the unshifted design.
// t phenotypes: W = [X~_L | Y~] (q + t columns); b holds p x ncols per
// phenotype, phenotype k at b + k * bstride (bstride 0: p * ncols).
cudaError_t launch_reduce_solve(const void* Xt, XtKind kind, int64_t ldt, int rows, const double* W,
                                int64_t ldw, const SolveConsts* sc, int q, int ncols, double* b, double* se,
                                int* status, cudaStream_t s, const float* W32 = nullptr,
                                const int8_t* shift = nullptr, DevStatus* st = nullptr, int num_sms = 0,
                                const CUtensorMap* xmap = nullptr, int t = 1, int64_t bstride = 0);
// Opt-in shared memory of the TMA-fed FP32 reduction (called once per split
// context).  With st, num_sms and xmap (a tiled map of the FP32 X~ buffer:
// dims {rows, columns}, box {RED_BOX_ROWS, RED_BOX_COLS}, no swizzle) given,
// launch_reduce_solve streams X~ through it: one persistent block per SM,
// bounded waits reporting into st.
constexpr int RED_BOX_ROWS = 256, RED_BOX_COLS = 32;
// The per-SNP sums formed by the inverse form's epilogue (tc::partials): their
// FP64 totals over the row groups, then the solve (q + t <= 8).
cudaError_t launch_partials_solve(const float* red, int ngroups, int64_t ldr, const SolveConsts* sc, int q, int t,
                                  int ncols, double* b, double* se, int* status, const int8_t* shift,
                                  cudaStream_t s, int64_t bstride = 0);
cudaError_t prepare_reduce_solve();
int w32_stride(int q);  // q + 1 columns (pass q + t - 1 for t phenotypes)
cudaError_t launch_make_w32(const double* W, int64_t ldw, int rows, int q, float* W32, cudaStream_t s);

// a11: per-SNP adjoint (chi2, d chi2/dh, y-weights), their sums over SNPs and
// the y-gradient; FP64.  GH = What^T What, What = [X^_L | y^] = L^-T W.
cudaError_t launch_adjoint(const double* Xt, const double* Xh, int64_t ldt, int rows, int n, const double* W,
                           const double* Wh, int64_t ldw, const SolveConsts* sc, const double* GH, int q,
                           int ncols, double h, double sigma2, double* chi2, double* dh, double* wv, double* uT,
                           double* dh_accum, double* dy_accum, double* dy_part, cudaStream_t s);
// Scratch of the y-gradient: adjoint_dy_chunks(bs) x n doubles (dy_part).
int adjoint_dy_chunks(int bs);
// Exact integer products of sliced M^-1 on the tensor cores (exact_products.cu),
// in two uses.  The split precisions' adjoint in its M^-1 form: W = M^-1
// (n_pad x n_pad FP64, symmetric, zero on the padding; the state takes
// ownership), What = [X^_L | y^] and W2 = W What (n_pad x (q+1) each, read
// during set-up only).  The sliced solve (GWAS_SLICED64): W (taken over and
// freed once sliced) and Wh = [X^_L | Y^] (n_pad x nw, nw = q + t, read during
// set-up only).  center: X_L[:, 0] is the intercept (SNP columns are shifted
// by their integer mean).
struct ExactProducts;
cudaError_t exact_adjoint_create(ExactProducts** out, double* W, const double* What, const double* W2, int n,
                                 int n_pad, int q, int bs, bool center, int num_sms, cudaStream_t s,
                                 int64_t* launches);
cudaError_t exact_solve_create(ExactProducts** out, double* W, const double* Wh, int nw, int n, int n_pad, int q,
                               int bs, bool center, int num_sms, cudaStream_t s, int64_t* launches);
// One block of ncols <= bs int8 SNP columns (device, any alignment): chi2 and
// d chi2/dh per SNP, wv (p per SNP), dh_accum += the block's sum of d chi2/dh,
// uT = the block's sums of wv[0..q-1], dy_accum += the block's y-gradient.
cudaError_t exact_adjoint_block(ExactProducts* E, const int8_t* X, int64_t ldx, int ncols, const SolveConsts* sc,
                                const double* GH, const double* What, double h, double sigma2, double* chi2,
                                double* dh, double* wv, double* uT, double* dh_accum, double* dy_accum,
                                DevStatus* st, cudaStream_t s, int64_t* launches);
// One block of the sliced solve in two steps: the cast of x' and the exact
// product (two launches; k0/k1, may be null, recorded around the product
// kernel), then the per-SNP sums and solve: b (t blocks of p x ncols), se,
// status.
cudaError_t exact_solve_product(ExactProducts* E, const int8_t* X, int64_t ldx, int ncols, DevStatus* st,
                                cudaStream_t s, cudaEvent_t k0, cudaEvent_t k1);
cudaError_t exact_solve_sums(ExactProducts* E, int ncols, const SolveConsts* sc, int t, double* b, double* se,
                             int* status, cudaStream_t s);
void exact_destroy(ExactProducts* E);
// CTAs of a full launch of the exact product kernel (2-SM clusters).
int exact_max_ctas(const ExactProducts* E);
// The sliced solve's slices of T (the product kernel and the per-SNP sums must
// agree): SLICED_SLABS integer slices of SLICED_BITS bits, every entry of a
// slice within +-2^(SLICED_BITS - 1) (exact in FP16).  The adjoint's slices of
// W are three of 10 bits (exact_products.cu, adjoint.cu).
constexpr int SLICED_SLABS = 4;
constexpr int SLICED_BITS = 11;
// The sliced solve's per-SNP sums from the exact products and the FP64 p x p
// solve (reduce_solve.cu).  C: slabs x RS rows per SNP (leading dimension
// ldc; only rows >= r_lo of the square part and the appended rows are read),
// acc: the product kernel's sums over the rows below r_lo (slabs x ldacc
// int64), xc: x' in FP16 (leading dimension ldx = n_pad), ne = q + t appended rows.
cudaError_t launch_sliced_solve(const int32_t* C, int64_t ldc, int RS, const long long* acc, int ldacc, int r_lo,
                                const __half* xc, int64_t ldx, int n, int ne, const double* inv_scale, const SolveConsts* sc, int q, int t, int ncols,
                                double* b, double* se, int* status, const int8_t* shift, cudaStream_t s,
                                int64_t bstride = 0);
// The per-SNP sums and adjoint from the exact products (adjoint.cu), then the
// block's sums of d chi2/dh (added to dh_accum) and of wv[0..q-1] (into uT).
cudaError_t launch_exact_adjoint_sums(const int32_t* C, int64_t ldc, int RS, const __half* xc, int64_t ldx, int n,
                                      int n_pad, int ne, const double* inv_scale, const SolveConsts* sc,
                                      const double* GH, int q, int ncols, double h, double sigma2, const int* xmax,
                                      double* chi2, double* dh, double* wv, double* dh_accum, double* uT,
                                      cudaStream_t s);
// 2-bit packed SNP columns (host_pack.cu): host packing of int8 columns whose
// values all lie in 0..3 (false otherwise), and the device unpacking into an
// int8 slot (leading dimension ldx, a multiple of 16, 16-byte aligned; rows
// n .. 16 ceil(n/16) - 1 written as 0).
bool pack2_columns(const int8_t* X, int64_t ldx, int n, int c0, int c1, uint8_t* P, int64_t ldp);
// Whether this host packs with AVX-512 (BW, VL), fast enough to pay inside the
// int8 stream; and a pool of persistent host threads (one per core with the
// caller) packing a block's columns in parallel (false: a value outside 0..3).
bool host_pack_fast();
struct PackPool;
PackPool* pack_pool_create();
bool pack_pool_run(PackPool* p, const int8_t* X, int64_t ldx, int n, int ncols, uint8_t* P, int64_t ldp);
void pack_pool_destroy(PackPool* p);
cudaError_t launch_unpack2(const uint8_t* P, int64_t ldp, int n, int ncols, int8_t* X, int64_t ldx, cudaStream_t s);
cudaError_t launch_log_diag(const double* L, int64_t ld, int n, double* out, cudaStream_t s);
cudaError_t launch_col_sumsq(const double* X, int64_t ld, int n, int ncols, double* out, cudaStream_t s);
cudaError_t launch_identity_cols(double* E, int n, int c0, int ncols, cudaStream_t s);
cudaError_t launch_null_residual(const double* W, int64_t ldw, int rows, int q, const SolveConsts* sc, double* R,
                                 cudaStream_t s);

// Read-only view of a context's study data and stream, for entry points that
// live outside the context's own file.
struct CtxView {
  int dev, num_sms, n, q, n_pad, P;
  int t;  // phenotypes
  cudaStream_t stream;
  const double* Aop;
  const double* W;
  const SolveConsts* sc;
  DevStatus* st;
  int64_t* launches;
  void* static_scratch;  // device address of the library's fixed scratch array on this device
};
bool ctx_view(gwas_ctx* ctx, CtxView* v);

// Set-up of the no-allocation block solve (static_scratch.cu), run by
// gwas_init with the context's device current: looks up the device address
// of the fixed scratch array (which loads its module, so the array is set
// aside now, not at the first solve) and loads the kernels that solve uses.
cudaError_t static_scratch_setup(void** addr);
// Load the FP64 solve's int8 kernel and the FP64 reduction kernel (lazy
// module loading would otherwise load them, allocating device memory for
// their code, at their first launch).
cudaError_t preload_trsm_f64_int8();
cudaError_t preload_reduce_solve_f64();

// Makes `dev` the calling thread's current device for the scope and gives the
// caller's device back on exit, so that a library call never leaves the
// calling thread on another device.
class DeviceScope {
 public:
  explicit DeviceScope(int dev) {
    if (cudaGetDevice(&prev_) != cudaSuccess) {
      cudaGetLastError();
      prev_ = -1;
    }
    err_ = prev_ == dev ? cudaSuccess : cudaSetDevice(dev);
  }
  ~DeviceScope() {
    int cur = -1;
    if (prev_ >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev_) cudaSetDevice(prev_);
  }
  DeviceScope(const DeviceScope&) = delete;
  DeviceScope& operator=(const DeviceScope&) = delete;
  cudaError_t status() const { return err_; }

 private:
  int prev_ = -1;
  cudaError_t err_ = cudaSuccess;
};

// The file reader over caller-owned pinned buffers (host_reader.cu).
int reader_open_with(gwas_reader** out, const char* path, int64_t offset, int64_t block_bytes, int64_t nblocks,
                     int64_t last_bytes, int depth, void* const* buffers);

}  // namespace gwas
