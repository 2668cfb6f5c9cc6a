/*
 * gwas_b300 — per-SNP generalized least squares (GLS) on one B300 GPU.
 *
 * C ABI of the library built from paper_1302_4332_b300/csrc (libgwas_b300.so).
 * Plain pointers and sizes only.  Every step of the computation runs in the
 * library's own CUDA kernels (sm_103a); there is no CPU fallback: without a
 * usable CUDA device every call that computes returns GWAS_ERR_CUDA.
 *
 * The computation (Beyer & Bientinesi, "Streaming Data from HDD to GPUs for
 * Sustained Peak Performance"):
 *
 *   Eq. 1    r_i = (X_i^T M^-1 X_i)^-1 X_i^T M^-1 y,   i = 1..m,
 *            X_i = (X_L | X_R_i)  (Sec. 1.3): X_L holds the p-1 fixed
 *            covariates, X_R_i is the i-th SNP column.
 *   Eq. 2    L L^T = M,  X~ = L^-1 X,  y~ = L^-1 y,
 *            r_i = (X~_i^T X~_i)^-1 X~_i^T y~.
 *   Listing 1: X~_L, y~, r_T = X~_L^T y~, S_TL = X~_L^T X~_L once; per SNP the
 *            triangular solve, S_BL = x~_i^T X~_L, S_BR = x~_i^T x~_i,
 *            r_B = x~_i^T y~ and the p x p SPD solve.
 *   Sec. 2.2 SNP columns are solved as blocks (trsv -> trsm).
 *
 * M = sigma2 (h Phi + (1 - h) I) with Phi the n x n kinship (the paper leaves
 * M's parametrisation open).  Each SNP result is r (called b here) with p
 * entries in the column order of X_i: entries 0..p-2 are the covariates, entry
 * p-1 the SNP effect; se_j = sqrt((S^-1)_jj), S = X_i^T M^-1 X_i.
 *
 * Storage: column-major.  Element (i, j) of an n-row matrix with leading
 * dimension ld is at [i + j * ld].
 *
 * Pointers: every array argument may be host memory (pageable or pinned) or
 * device memory of the context's device; the library finds out which with
 * cudaPointerGetAttributes.  When the SNP input and all outputs are device
 * pointers the call is asynchronous on the context's stream and device-side
 * errors surface at the next gwas_synchronize(); otherwise the call returns
 * once the outputs are in host memory.  All pointers are borrowed for the
 * duration of the call only; inputs to gwas_init are copied.
 *
 * Errors: every int-returning call returns GWAS_OK (0) or a negative
 * GWAS_ERR_* code; gwas_strerror() names it and gwas_last_error_detail()
 * gives the context's last message.  A SNP whose design is numerically
 * collinear (last pivot d^2 <= 1e-7 * S_BR, e.g. a monomorphic SNP) is not a
 * call error: its status is GWAS_SNP_SINGULAR and its b and se are NaN.
 */
#ifndef GWAS_B300_H
#define GWAS_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GWAS_OK 0
#define GWAS_ERR_ARG (-1)        /* bad n, p, h, sigma2, size, leading dimension, or NULL pointer */
#define GWAS_ERR_NOT_SPD (-2)    /* Cholesky pivot <= 0 (index: gwas_not_spd_index) or S_TL singular */
#define GWAS_ERR_CUDA (-3)       /* CUDA runtime/driver error, or no usable device */
#define GWAS_ERR_TIMEOUT (-4)    /* a bounded device-side or host-side wait ran out */
#define GWAS_ERR_IO (-5)         /* host-side input/output failure */
#define GWAS_ERR_NOMEM (-6)      /* device or pinned-host allocation failed */
#define GWAS_ERR_UNSUPPORTED (-7)/* a configuration the library was compiled without */

#define GWAS_SNP_OK 0
#define GWAS_SNP_SINGULAR 1

/* Arithmetic of the blocked triangular solve X~ = L^-1 X_R (Sec. 2.2's trsm).
 * The Cholesky of M, the diagonal-block inverses of L, X~_L / y~ and the
 * p x p solves are FP64 in every mode.
 *   GWAS_FP64   : all of the solve in FP64.
 *   GWAS_TF32X3 : block products on the tensor cores, each FP32 operand split
 *                 into TF32 hi + lo, three products (hi*hi + hi*lo + lo*hi),
 *                 FP32 accumulation.
 *   GWAS_BF16X3 : the same with BF16 hi + lo pieces.
 *   (In the inverse tile mode the dosages are exact, so hi*X + lo*X: two products.)
 *   GWAS_F16X2  : inverse tile mode only (tile_mode AUTO or INVERSE; others return
 *                 GWAS_ERR_ARG): each row of L^-1 is scaled by a power of two so its
 *                 largest entry lies in [2^13, 2^14), then split into FP16 hi + lo
 *                 (11 + 11 significant bits against BF16's 8 + 8), the dosages exact
 *                 in FP16: two products at the BF16 rate; results scaled back exactly.
 *   GWAS_SLICED64 : FP64-class results (the FP64 path's tolerance) from the tensor cores.
 *                 Eq. 1's X_i^T M^-1 X_i and X_i^T M^-1 y are formed with W = M^-1 made
 *                 explicit once in FP64 (L^-T L^-1, at gwas_init): per SNP, with x' the
 *                 int8 column shifted by its integer mean, x'^T [X^_L | y^] (X^_L = W X_L,
 *                 y^ = W y) and x'^T W x' = 2 x'^T T x' (T = W's lower triangle, diagonal
 *                 halved).  T's rows (one power-of-two scale) are cut into four 11-bit
 *                 integer slices (entries within +-1024) and [X^_L | y^]'s columns into
 *                 six, each exact in FP16; every slice times the int8 dosages is an exact
 *                 integer (FP16 products, FP32 accumulation kept at most 2^24), so the
 *                 only error is T's 44-bit representation.  Four triangular FP16 products
 *                 per block.  Tile modes, strip_group, separate_sums and single_piece do
 *                 not apply (GWAS_ERR_ARG if set); batches take split contexts only.  A
 *                 block whose largest |x - c| * 1024 * n_pad reaches 2^31 is refused
 *                 (GWAS_ERR_ARG; never for dosages 0..2 below n = 1,000,000; any int8
 *                 values up to n = 8,192).  Set-up takes 16 n_pad^2 bytes for a while (W
 *                 and the transpose operator), the context keeps 8 n_pad^2 (slices) +
 *                 16 n_pad bs (products) bytes beside the FP64 study data. */
typedef enum { GWAS_FP64 = 0, GWAS_TF32X3 = 1, GWAS_BF16X3 = 2, GWAS_F16X2 = 3, GWAS_SLICED64 = 4 } gwas_precision;

typedef struct {
  int precision;   /* gwas_precision */
  int bs;          /* SNP columns per block: the most columns one solve call takes (>= 1) */
  int ring_depth;  /* device slots of the host->device block ring used by gwas_solve_stream (>= 2) */
  int device;      /* CUDA device ordinal; -1 = the current device */
  int strip_group; /* split modes: tiles are handed out row panel by row panel over groups of this
                      many 256-column strips (0 = all strips of the block at once); smaller groups keep
                      the strips being re-read inside the L2 */
  int tile_mode;   /* split modes, how the solve's tiles map onto the SMs:
                      GWAS_TILES_AUTO (0, default): the measured fastest of the others for the split;
                      GWAS_TILES_SINGLE (1): every 128-row tile on its own SM;
                      (2 is not a mode: GWAS_ERR_ARG)
                      GWAS_TILES_PAIR_MMA (3): panels 2u and 2u+1 as one 256-row tensor-core product
                        on the two SMs of a cluster;
                      GWAS_TILES_INVERSE (4): L^-1 is formed once at gwas_init (the FP64 blocked
                        solve of the identity, n^3/3 flop) and split like the block operator; a
                        block is then the triangular product L^-1 X_R with no dependency between its
                        tiles (256-row products on 2-SM clusters, longest first).  Costs one
                        n_pad x bs cast copy of the block and, at set-up, up to 16 n_pad^2 bytes of
                        transient device memory (n_pad = n rounded up to 128) */
  int traits;      /* phenotypes t sharing the study (0 = 1): y is n x t column-major, W = [X~_L | Y~];
                      1 <= t <= 16 and p - 1 + t <= 16.  The solve of each SNP block is shared by the t
                      phenotypes; S (so se and status) does not depend on y, only b does: every b output
                      holds t consecutive p x ncols (or p x m) column-major blocks, phenotype k at
                      b + k p ncols.  Batches, the adjoint, REML and gwas_solve_block_static take t = 1
                      (else GWAS_ERR_UNSUPPORTED) */
  int separate_sums; /* inverse tile mode (with p - 1 + t <= 8): 0 (default) forms the per-SNP sums
                        x~ . [X~_L | Y~] and x~ . x~ in the solve's epilogue, which then stores no X~
                        (FP32 partial sums per row panel, added by a small pass as double-FP32 pairs
                        before the FP64 p x p solves); 1 stores X~ and sums it in a separate pass.
                        Other modes and sizes always use the separate pass */
  int single_piece;  /* precision studies only (inverse tile mode): 1 keeps L^-1 as its hi piece alone
                        (its lo piece zeroed: one BF16, TF32 or row-scaled FP16 rounding of L^-1);
                        b and se then carry that rounding, far above the split forms' 1e-5 */
  int stream_pack;   /* how gwas_solve_stream moves int8 host columns to the device: -1 (default) packs
                        each block whose values all lie in 0..3 into 2-bit codes on the host (the
                        encoding of gwas_pack_dosages2; a quarter of the link's bytes, unpacked on the
                        GPU) when the host CPU has AVX-512 (BW, VL), where a pool of host threads packs
                        faster than the link carries int8, and the solve outruns the int8 link (BF16x3
                        and F16x2 in the inverse tile mode), else copies int8; 0 always copies int8;
                        1 packs wherever the values allow.  A block with any other value crosses as int8.
                        Results are identical either way.  The pool (one thread per host core, created
                        on the first packed call) and ring_depth pinned host slots of ceil(n/4)
                        (rounded up to 16) x bs bytes belong to the context */
} gwas_config;

enum {
  GWAS_TILES_AUTO = 0,
  GWAS_TILES_SINGLE = 1,
  GWAS_TILES_PAIR_MMA = 3,
  GWAS_TILES_INVERSE = 4
};

typedef struct gwas_ctx gwas_ctx; /* opaque; owned by the library */

/* Fills *cfg with the defaults: GWAS_FP64, bs = 4096, ring_depth = 3, device -1. */
void gwas_config_default(gwas_config *cfg);

/* Sets up one study (Listing 1, loop-invariant part; Sec. 3: L stays on the GPU).
 *   n       samples (>= 1); p columns of each X_i (1 <= p <= 16)
 *   phi_or_L n x n, leading dimension n.  is_L = 0: the kinship Phi (symmetric;
 *           only its lower triangle is read) and M = sigma2 (h Phi + (1-h) I)
 *           is formed on the device; is_L = 1: the lower Cholesky factor L of M
 *           (upper triangle ignored; h and sigma2 are then only recorded).
 *   XL      n x (p-1) covariates, leading dimension n (may be NULL when p = 1)
 *   y       n phenotypes
 *   h       0 <= h <= 1;  sigma2 > 0
 *   cfg     NULL for the defaults
 *   stream  cudaStream_t the context issues its work on (NULL: the legacy default stream)
 * On success *out owns device memory of about 8 n^2 bytes (FP64 L and the
 * block operator) plus, for the split modes, 4 n^2 bytes of split copies,
 * plus per-block scratch of about 8 n bs bytes.
 * Errors: GWAS_ERR_ARG, GWAS_ERR_NOT_SPD (M or S_TL not positive definite),
 * GWAS_ERR_NOMEM, GWAS_ERR_CUDA, GWAS_ERR_UNSUPPORTED. */
int gwas_init(gwas_ctx **out, int n, int p, const double *phi_or_L, int is_L, const double *XL,
              const double *y, double h, double sigma2, const gwas_config *cfg, void *stream);

/* One block of SNPs (Listing 1 loop body, batched per Sec. 2.2).
 *   XR      n x ncols int8 dosages, leading dimension ldx >= n (rows >= n ignored)
 *   ncols   0 <= ncols <= cfg.bs
 *   b, se   p x ncols FP64 outputs, leading dimension p (se may be NULL)
 *   status  ncols ints, GWAS_SNP_OK / GWAS_SNP_SINGULAR (may be NULL)
 * Errors: GWAS_ERR_ARG, GWAS_ERR_CUDA, GWAS_ERR_TIMEOUT. */
int gwas_solve_block(gwas_ctx *ctx, const int8_t *XR, int64_t ldx, int ncols, double *b, double *se,
                     int *status);

/* As gwas_solve_block with FP64 SNP values (any real dosages). */
int gwas_solve_block_f64(gwas_ctx *ctx, const double *XR, int64_t ldx, int ncols, double *b, double *se,
                         int *status);

/* Whole-study streaming (Sec. 3.1, re-designed): m SNP columns in HOST memory
 * are cut into blocks of cfg.bs columns and copied into a ring of
 * cfg.ring_depth device slots on a copy stream, overlapping the solve of the
 * previous blocks on the compute stream; results are copied back per block.
 * With cfg.stream_pack (see gwas_config) a block whose values all lie in 0..3
 * is packed to 2-bit codes by host threads and crosses the link in a quarter
 * of the bytes; results are the same either way.
 *   XR_host n x m int8, leading dimension ldx >= n (pinned memory gives full
 *           link speed; pageable memory works through the driver's staging)
 *   b_host, se_host p x m;  status_host m (se_host / status_host may be NULL)
 * Errors: GWAS_ERR_ARG, GWAS_ERR_CUDA, GWAS_ERR_TIMEOUT, GWAS_ERR_NOMEM (the
 * packing slots or threads could not be made).
 * Returns when all results are in host memory. */
int gwas_solve_stream(gwas_ctx *ctx, const int8_t *XR_host, int64_t ldx, int64_t m, double *b_host,
                      double *se_host, int *status_host);

/* gwas_solve_stream over SNP columns held 2-bit packed in HOST memory (hard
 * calls 0..3, four to a byte, as gwas_pack_dosages2 writes them and as genotype
 * files commonly store them): the host link carries ceil(n/4) bytes per SNP
 * instead of n.  The split inverse form's cast pre-pass reads the codes as
 * they are (n <= 16384); otherwise a kernel unpacks each block into the
 * device ring slot first.  Results are those of gwas_solve_stream on the
 * unpacked int8 columns; bits of rows past n are ignored.
 *   P_host  ceil(n/4) bytes per column, leading dimension ldp >= ceil(n/4)
 * Other arguments, errors and results as gwas_solve_stream.  (Packing inside
 * the stream pays only on a host whose cores pack faster than the link carries
 * int8: with AVX-512 16 cores pack ~73 GB/s, the scalar form ~20 GB/s, the
 * link ~56 GB/s; gwas_config.stream_pack chooses.) */
int gwas_solve_stream_packed(gwas_ctx *ctx, const uint8_t *P_host, int64_t ldp, int64_t m, double *b_host,
                             double *se_host, int *status_host);

/* The 2-bit encoding of gwas_solve_stream_packed (a storage format): column c
 * of the n x ncols int8 array X (leading dimension ldx) becomes P[c ldp ..
 * c ldp + ceil(n/4) - 1], byte k holding X[4k + i, c] in bits 2i .. 2i+1
 * (i = 0..3; rows past n as 0); ldp >= ceil(n/4).  Host memory, host code.
 * Returns GWAS_ERR_ARG (P then undefined) if a value lies outside 0..3. */
int gwas_pack_dosages2(const int8_t *X, int64_t ldx, int n, int ncols, uint8_t *P, int64_t ldp);

/* Bytes the context has copied host -> device for SNP blocks since gwas_init
 * (the block solves with host input and both streams; packed columns count
 * their packed bytes). */
int64_t gwas_h2d_bytes(const gwas_ctx *ctx);

/* gwas_solve_block without any allocation, FP64 solve only.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory when they solve -- e.g. a process whose device memory is
 * held by another framework's caching allocator, or a service that must not
 * call cudaMalloc once it is serving.  They run gwas_init once at start-up;
 * this call then allocates nothing (no cudaMalloc, no cudaFree, no library
 * routine that allocates).
 *   XR, b, se, status: DEVICE pointers only (host pointers: GWAS_ERR_ARG);
 *   layouts and outputs as gwas_solve_block; asynchronous on the context's
 *   stream (device-side errors surface at gwas_synchronize).
 * Scratch: one fixed device array of GWAS_STATIC_SCRATCH_BYTES inside the
 * library.  gwas_init, with the context's device current, looks the array's
 * device address up (cudaGetSymbolAddress) and keeps it in the context; that
 * lookup loads the array's module, which is when CUDA sets the array aside on
 * the device (it stays until the process exits), and gwas_init also loads the
 * kernels this call launches -- so every context holds its device's share of
 * the array from gwas_init on, and the call itself needs no device memory even
 * when the device's memory is full.  A call needs
 *   256-byte-rounded (128 + 4 * ceil(n/128) * ceil(ncols/64)) + 8 * n_pad * ncols
 * bytes, n_pad = n rounded up to 128 (at n = 10,000: up to 414 columns); a
 * larger call returns GWAS_ERR_ARG before anything is launched.  Every call
 * uses the same array and it keeps the previous call's contents (the call
 * clears what must start at zero): calls whose GPU work overlaps -- two
 * streams, or two contexts at once -- race on it and give wrong results.
 * The call runs the FP64 solve whatever the context's precision.
 * Errors: GWAS_ERR_ARG, GWAS_ERR_CUDA. */
#define GWAS_STATIC_SCRATCH_BYTES (32u * 1024u * 1024u)
int gwas_solve_block_static(gwas_ctx *ctx, const int8_t *XR, int64_t ldx, int ncols, double *b, double *se,
                            int *status);

/* The differentiation form (not in the paper): for one block of SNPs, the
 * Wald statistic chi2_i = b_{p-1}^2 / (S^-1)_{p-1,p-1} of every SNP and the
 * gradient of their sum with respect to h and y; needs 0 < h <= 1 (it uses
 * dM/dh = (M - sigma2 I) / h).
 *   GWAS_FP64 contexts: forward solve X~ = L^-1 X and transpose solve
 *     X^ = L^-T X~ = M^-1 X in FP64, then per-SNP p x p adjoints.  The first
 *     call builds the transpose operator (8 n^2 bytes).
 *   Split contexts (any precision and tile mode): every per-SNP input from one
 *     exact integer product on the tensor cores -- M^-1 (formed in FP64 at the
 *     first call, 8 n^2 bytes, plus three FP16 slices of it, 6 n^2 bytes) and
 *     the solved covariates and phenotype, sliced into 10-bit integer pieces,
 *     times the block's int8 dosages with FP32 accumulation kept below 2^24 --
 *     then the same FP64 adjoint arithmetic: results agree with the FP64 path
 *     to ~1e-8.  A block whose largest |x - c| times 512 n_pad reaches 2^31
 *     (never for dosages 0..2 below n = 2,000,000) is refused: GWAS_ERR_ARG.
 *   chi2, dchi2_dh  ncols each, may be NULL (a collinear SNP: NaN and 0)
 *   dh_accum        one double; the block's sum of d chi2/dh is ADDED to it
 *   dy_accum        n doubles; the block's d(sum chi2)/dy is ADDED to it
 * Host or device pointers.  Errors: GWAS_ERR_ARG, GWAS_ERR_CUDA, GWAS_ERR_TIMEOUT. */
int gwas_adjoint_block(gwas_ctx *ctx, const int8_t *XR, int64_t ldx, int ncols, double *chi2, double *dchi2_dh,
                       double *dh_accum, double *dy_accum);

/* REML of the null model y ~ N(X_L beta, s2 (h Phi + (1 - h) I)) with s2
 * profiled out (q = p - 1 covariates), evaluated on the GPU in FP64 at one h:
 *   out[0] = l(h) = -1/2 [ (n - q) log s2 + log|V| + log|X_L^T V^-1 X_L| ]
 *   out[1] = dl/dh = (tr(P) - ||P y||^2 / s2) / (2 h),   out[2] = s2,
 * P = V^-1 - V^-1 X_L (X_L^T V^-1 X_L)^-1 X_L^T V^-1, s2 = y^T P y / (n - q).
 * phi n x n, XL n x q, y n (host or device).  0 < h <= 1. */
int gwas_reml_eval(int n, int q, const double *phi, const double *XL, const double *y, double h,
                   const gwas_config *cfg, void *stream, double *out);

/* Gradient-based REML fit of h from h0 (0 < h0 < 1): the sign change of
 * dl/dh is bracketed by stepping uphill, then closed by modified regula
 * falsi until the bracket is narrower than tol (or max_evals likelihood
 * evaluations were spent).  *h_out, *loglik_out (may be NULL), *evals_out
 * (may be NULL). */
int gwas_reml_fit(int n, int q, const double *phi, const double *XL, const double *y, double h0, double tol,
                  int max_evals, const gwas_config *cfg, void *stream, double *h_out, double *loglik_out,
                  int *evals_out);

/* The batching form (not in the paper): several studies -- each its own
 * context (own n, factor and operator), all in the same split precision on
 * the same device -- solved by ONE persistent tensor-core launch whose tiles
 * come from all studies, row panel by row panel (or study after study), so
 * small studies never leave SMs idle.  The whole step (shift pre-passes, the
 * batched launch, every study's reductions) is captured into a CUDA graph on
 * first use and replayed; a new ncols vector or tile order re-captures it.
 * At most 8 studies. */
typedef struct gwas_batch gwas_batch;
int gwas_batch_create(gwas_batch **out, gwas_ctx *const *studies, int nstudies, void *stream);
/* XR[i] n_i x ncols[i] int8 (leading dimension ldx[i], host or device), ncols[i] <= bs of
 * study i (0 skips it); b[i], se[i] p x ncols[i]; status[i] ncols[i] (se, status and
 * their entries may be NULL).  Inputs are copied into the batch's fixed device slots;
 * asynchronous on the batch stream when every pointer is device memory. */
int gwas_batch_solve(gwas_batch *B, const int8_t *const *XR, const int64_t *ldx, const int *ncols,
                     double *const *b, double *const *se, int *const *status);
int gwas_batch_synchronize(gwas_batch *B);
/* 0: interleave the studies row panel by row panel (default); 1: one study after another. */
int gwas_batch_set_order(gwas_batch *B, int order_mode);
/* k blocks per study in one graph replay: the captured graph holds k steps
 * (each: the pre-passes, one batched launch over all studies, every study's
 * reductions), so one cudaGraphLaunch solves k blocks of every study.
 * Arrays are indexed [j * nstudies + i] (study i's j-th block); otherwise as
 * gwas_batch_solve.  1 <= k <= GWAS_BATCH_MAX_STEPS; the batch keeps k sets
 * of device slots once used. */
#define GWAS_BATCH_MAX_STEPS 16
int gwas_batch_solve_k(gwas_batch *B, int k, const int8_t *const *XR, const int64_t *ldx, const int *ncols,
                       double *const *b, double *const *se, int *const *status);
/* Autotuner.  Candidates: SNP columns per study per launch (512, 1024, ... up
 * to the smallest bs); the tile mode -- the studies' own and, for BF16x3 and
 * TF32x3 batches, the other of GWAS_TILES_INVERSE and GWAS_TILES_PAIR_MMA
 * (their operators are built once for the trial, kept if chosen); the
 * inverse form's operand depth in 64-byte K-steps (8 or 6, two steps to a
 * shared-memory stage); the substitution's tile order
 * (interleaved, or study after study over all strips or groups of 8 or 4).
 * Each candidate is timed (CUDA events; one warm-up, then reps) as whole
 * gwas_batch_solve steps with device arrays on seeded dosage blocks
 * (Binomial(2, f), f in [0.05, 0.5), generated on the device) -- the work of
 * a real step, including its input and output copies.  The fastest is kept
 * for later solves. */
typedef struct {
  int cols;           /* SNP columns per study per launch */
  int tile_mode;      /* GWAS_TILES_INVERSE or GWAS_TILES_PAIR_MMA */
  int stages;         /* operand depth of the inverse-form kernel in K-steps (8 or 6; two a stage) */
  int order;          /* 0 interleaved, 1 study after study */
  int strip_group;    /* 0 = all strips */
  double snps_per_s;  /* the chosen candidate's rate over all studies */
} gwas_batch_tuning;
int gwas_batch_autotune_ex(gwas_batch *B, int reps, gwas_batch_tuning *out);
/* The same, reporting the columns, order and rate only. */
int gwas_batch_autotune(gwas_batch *B, int reps, int *cols_out, int *order_out, double *snps_per_s_out);
/* The batching form out of core (Sec. 3.1's disk -> main memory -> GPU, for several studies):
 * study i's int8 dosages are columns col0[i] .. col0[i]+m[i]-1 of the file paths[i] (n_i rows,
 * column-major, leading dimension ldx[i] bytes after header_bytes[i]).  One reader thread per
 * study prefetches blocks of `cols` columns (1 <= cols <= every study's bs) into three pinned host
 * buffers; each step copies one block per study into the batch's device slots and replays the
 * captured batched launch, while the readers fetch the next blocks.  A study whose columns are
 * done drops out of the later steps.  Results: b_host[i] (p_i x m[i], column-major), se_host[i]
 * and status_host[i] (may be NULL, as may the arrays of them).  Errors: GWAS_ERR_IO (open, read,
 * file too short), GWAS_ERR_TIMEOUT (no block within 120 s), and those of gwas_batch_solve. */
int gwas_batch_solve_files(gwas_batch *B, const char *const *paths, const int64_t *header_bytes, const int64_t *ldx,
                           const int64_t *col0, const int64_t *m, int cols, double *const *b_host,
                           double *const *se_host, int *const *status_host);
/* The same over files of 2-bit packed columns (gwas_pack_dosages2's encoding: ceil(n_i/4) bytes a
 * column, leading dimension ldp[i] >= ceil(n_i/4) bytes after header_bytes[i]): a quarter of the
 * int8 file's bytes from disk and over the host link; each step's packed blocks are copied into a
 * device staging area (ceil(n_i/4) rounded up to 16 bytes x bs per study, allocated on first use)
 * and expanded into the batch's int8 slots on the GPU before the replay, so the results equal
 * gwas_batch_solve_files on the int8 file bit for bit.  Bits of rows past n_i are ignored.
 * Errors: those of gwas_batch_solve_files; GWAS_ERR_ARG also for ldp[i] < ceil(n_i/4). */
int gwas_batch_solve_files_packed(gwas_batch *B, const char *const *paths, const int64_t *header_bytes,
                                  const int64_t *ldp, const int64_t *col0, const int64_t *m, int cols,
                                  double *const *b_host, double *const *se_host, int *const *status_host);
int64_t gwas_batch_kernel_launches(const gwas_batch *B);
const char *gwas_batch_last_error_detail(const gwas_batch *B);
void gwas_batch_destroy(gwas_batch *B);

/* Out-of-core streaming from a file (Sec. 3.1: disk -> main memory -> GPU).
 * The file holds n x M int8 dosages, column-major with leading dimension ldx
 * bytes, after header_bytes; columns col0 .. col0+m-1 are solved (so a run
 * can resume from a column cursor).  A reader thread prefetches blocks of
 * cfg.bs columns into three pinned host buffers while earlier blocks are
 * copied into the device ring and solved; results go to b_host, se_host,
 * status_host (p x m, p x m, m; the last two may be NULL).
 * Errors: GWAS_ERR_IO (open failure, read error, file too short),
 * GWAS_ERR_TIMEOUT (no block within 120 s), and those of gwas_solve_block. */
int gwas_solve_file(gwas_ctx *ctx, const char *path, int64_t header_bytes, int64_t ldx, int64_t col0, int64_t m,
                    double *b_host, double *se_host, int *status_host);

/* Disk to disk, resumable (Sec. 3.1's streaming with the results written back):
 * columns col0 .. col0+m-1 of the dosage file, as in gwas_solve_file, with the
 * results of column col0 + j written to out_path as record j:
 *   out_path = a 64-byte header, then m records of GWAS_RESULT_RECORD_BYTES(p) bytes;
 *   header: char magic[8] = "GWASRES\0", uint32 version (1), uint32 p, uint64 n,
 *           uint64 col0, uint64 m, uint32 record_bytes, uint32 precision, 16 bytes 0;
 *   record: double b[p], double se[p], int32 status, int32 0 (little-endian).
 * A checkpoint file out_path + ".ckpt" (the same header with magic "GWASCKP\0"
 * and, at byte 48, uint64 done) advances every 16 blocks and at the end, each
 * time after the records it covers were flushed to disk (fdatasync).  With
 * flags & GWAS_PACKED_INPUT: the input columns are 2-bit packed (the encoding
 * of gwas_pack_dosages2, ldx >= ceil(n/4) bytes per column): a quarter of the
 * bytes from disk and over the link, unpacked on the GPU; results identical.
 * flags & GWAS_RESUME the run continues from the checkpoint's `done` column
 * (rewriting at most the blocks after it; a missing checkpoint starts at 0); a
 * checkpoint of another run (p, n, col0, m, precision) is GWAS_ERR_ARG.
 * *done_out (may be NULL) = the columns on disk when the call returns.
 * Errors: GWAS_ERR_IO (the input as in gwas_solve_file; creating or writing the
 * output or checkpoint), and those of gwas_solve_file. */
#define GWAS_RESUME 1
#define GWAS_PACKED_INPUT 2
#define GWAS_RESULT_RECORD_BYTES(p) (16 * (p) + 8)
/* With t phenotypes a record holds double b[t][p] (phenotype-major), se[p], status, 0; the header
 * stores t at byte 56 (uint64). */
#define GWAS_RESULT_RECORD_BYTES_T(p, t) (8 * (p) * ((t) + 1) + 8)
int gwas_solve_file_out(gwas_ctx *ctx, const char *in_path, int64_t header_bytes, int64_t ldx, int64_t col0,
                        int64_t m, const char *out_path, int flags, int64_t *done_out);

/* The prefetching file reader on its own: blocks of block_bytes bytes (the
 * last one last_bytes, 0 = full) from `offset`, read by a host thread into
 * `depth` >= 2 pinned buffers ahead of the consumer.  gwas_reader_next waits
 * (at most timeout_ms) for the next block in file order; its buffer stays
 * valid until the matching gwas_reader_release (oldest first). */
typedef struct gwas_reader gwas_reader;
int gwas_reader_open(gwas_reader **out, const char *path, int64_t offset, int64_t block_bytes, int64_t nblocks,
                     int64_t last_bytes, int depth);
int gwas_reader_next(gwas_reader *r, const void **buf, int64_t *bytes, int timeout_ms);
int gwas_reader_release(gwas_reader *r);
const char *gwas_reader_error_detail(const gwas_reader *r);
void gwas_reader_close(gwas_reader *r);

/* Waits for the context's queued work and reports device-side errors
 * (GWAS_ERR_TIMEOUT when a bounded wait inside a kernel gave up). */
int gwas_synchronize(gwas_ctx *ctx);

/* Sets the stream later calls are issued on (cudaStream_t; NULL = legacy default). */
int gwas_set_stream(gwas_ctx *ctx, void *stream);

/* Study facts: n, p, the padded row count of the device layout, precision. */
int gwas_get_info(const gwas_ctx *ctx, int *n, int *p, int *n_pad, int *precision, int *bs);

/* Launch shape of the blocked triangular solve for a full block: *ctas thread blocks (one per SM),
   in clusters of *cluster_size (2 in the pair tile modes, else 1), and *tile_mode, the resolved
   gwas_config.tile_mode (never GWAS_TILES_AUTO).  FP64 contexts report the occupancy-bound grid of
   the FP64 solve, 1 and GWAS_TILES_SINGLE; GWAS_SLICED64 contexts the exact product kernel's CTAs,
   2 and GWAS_TILES_AUTO (no tile mode applies).  Any output pointer may be NULL. */
int gwas_solve_shape(const gwas_ctx *ctx, int *ctas, int *cluster_size, int *tile_mode);

/* Index of the first failing Cholesky pivot after GWAS_ERR_NOT_SPD, else -1. */
int64_t gwas_not_spd_index(const gwas_ctx *ctx);

/* Device copy of the lower factor L (n x n, leading dimension ld >= n) into
 * caller memory (host or device); for checks of the factorization. */
int gwas_copy_factor(gwas_ctx *ctx, double *L, int64_t ld);

/* Stage timing with CUDA events recorded around each stage on the stream the
 * stage runs on; for measurement only (a few microseconds per event pair).
 * Stages: GWAS_STAGE_H2D (block copy in), GWAS_STAGE_TRSM (the blocked
 * triangular solve, with the split paths' cast or shift pre-pass),
 * GWAS_STAGE_REDUCE (reductions + p x p solves), GWAS_STAGE_D2H (results
 * out), GWAS_STAGE_SOLVE (the solve kernel's launch alone, inside
 * GWAS_STAGE_TRSM).  gwas_timing_enable(ctx, 1) clears and starts
 * the accumulators, 0 stops them.  gwas_timing_read waits for the recorded
 * events and writes the summed milliseconds and the number of timed launches
 * per stage into ms[GWAS_NSTAGES] and count[GWAS_NSTAGES]. */
#define GWAS_STAGE_H2D 0
#define GWAS_STAGE_TRSM 1
#define GWAS_STAGE_REDUCE 2
#define GWAS_STAGE_D2H 3
#define GWAS_STAGE_SOLVE 4
#define GWAS_NSTAGES 5
int gwas_timing_enable(gwas_ctx *ctx, int enable);
int gwas_timing_read(gwas_ctx *ctx, double *ms, int64_t *count);

/* Diagnostic of the device-side failure detection: one thread waits, bounded
 * by limit_us microseconds (1 .. 1,000,000) of %globaltimer, for something
 * that never happens -- kind 0: a device flag that nothing sets, kind 1: a
 * shared-memory mbarrier that nothing arrives on -- with the same bounded
 * wait, error word and abort flag as the solve kernels.  Returns
 * GWAS_ERR_TIMEOUT (the expected outcome: the wait ran out, the device
 * recorded it and the host read and cleared it) and leaves the context
 * usable; GWAS_ERR_ARG for a bad kind or limit. */
int gwas_check_timeout(gwas_ctx *ctx, int kind, int limit_us);

/* Kernel launches the context issued since it was created (all kinds). */
int64_t gwas_kernel_launches(const gwas_ctx *ctx);

const char *gwas_strerror(int code);
const char *gwas_last_error_detail(const gwas_ctx *ctx);

/* Frees everything the context owns.  NULL is accepted. */
void gwas_destroy(gwas_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* GWAS_B300_H */
