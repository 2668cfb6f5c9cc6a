// The C ABI of gwas_b300 (include/gwas_b300.h): study set-up, block solves and
// the host->device block stream.  Host code only orchestrates; every step of
// the computation is one of the library's kernels.
#include <cuda.h>
#include <cuda_runtime.h>

#include <fcntl.h>
#include <unistd.h>

#include <algorithm>
#include <cerrno>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "gwas_internal.cuh"
#include "tc_ptx.cuh"
#include "trsm_tc.cuh"

using namespace gwas;

struct gwas_ctx {
  int dev = 0;
  int num_sms = 148;
  cudaStream_t stream = nullptr;
  cudaStream_t copy_stream = nullptr;
  cudaStream_t out_stream = nullptr;  // the whole-study stream's result copies
  int n = 0, p = 0, q = 0, n_pad = 0, P = 0;
  int t = 1;  // phenotypes sharing the study (columns of y)
  int prec = GWAS_FP64, bs = 0, ring_depth = 0;
  double h = 0.0, sigma2 = 0.0;
  // study data (device)
  double* L = nullptr;     // n_pad x n_pad column-major
  double* Dinv = nullptr;  // P x TB x TB
  double* Aop = nullptr;   // n_pad x n_pad row-major block operator
  double* W = nullptr;     // n_pad x (q+1): [X~_L | y~]
  double* G = nullptr;     // (q+1)^2
  SolveConsts* sc = nullptr;
  DevStatus* st = nullptr;
  // per-block scratch (device)
  double* Xt = nullptr;    // n_pad x bs FP64 (FP64 mode; set-up in every mode)
  Sched* sched = nullptr;  // scheduler counter + tile flags
  size_t sched_bytes = 0;
  tc::TcState* tcs = nullptr;  // split-precision state (TF32X3 / BF16X3)
  float* W32 = nullptr;        // W in FP32, row-major (split-path reductions)
  bool intercept = false;      // X_L[:, 0] == 1 for every sample
  // adjoint form (built on first use)
  double* AopT = nullptr;      // transpose block operator, row-major
  double* Xhat = nullptr;      // n_pad x bs: X^ = L^-T X~
  double* What = nullptr;      // n_pad x (q+1): [X^_L | y^]
  double* GH = nullptr;        // (q+1)^2 Gram of What
  bool adjoint_ready = false;  // the arrays below are made and What / GH hold their values
  double* adj = nullptr;       // per-SNP chi2 (bs), dh (bs), y-weights (bs x p), uT (q), dh/dy staging (1 + n),
                               // the y-gradient's chunk partials (adjoint_dy_chunks(bs) x n)
  ExactProducts* exact = nullptr;   // split precisions: the adjoint's exact products (built on first use)
  ExactProducts* sliced = nullptr;  // GWAS_SLICED64: the solve's exact products (built at gwas_init)
  bool separate_sums = false, single_piece = false;  // the split set-up's options (a batch's tuner repeats them)
  // pinned host buffers of the file reader, kept across gwas_solve_file calls
  std::vector<void*> file_buf;
  int64_t file_buf_bytes = 0;
  // device staging for host arguments
  std::vector<int8_t*> ring;      // ring_depth slots of n_pad x bs int8
  std::vector<cudaEvent_t> ev_copied, ev_free, ev_out;
  double* d_b = nullptr;  // ring_depth x p x bs
  double* d_se = nullptr;
  int* d_status = nullptr;
  double* h_b = nullptr;  // pinned result staging, ring_depth slots
  double* h_se = nullptr;
  int* h_status = nullptr;
  double* f64_in = nullptr;  // n x bs FP64 staging for gwas_solve_block_f64 with host input
  // 2-bit packed input (gwas_solve_stream_packed; set up on its first call)
  int64_t ldp = 0;                   // packed bytes per column in a device slot (ceil(n/4) rounded up to 16)
  std::vector<uint8_t*> dpack;       // ring_depth device slots of ldp x bs bytes
  // int8 host columns packed by host threads in gwas_solve_stream (gwas_config.stream_pack;
  // the pool and the pinned slots are made on the first packed call)
  int stream_pack = 0;  // gwas_config.stream_pack: -1 auto, 0 off, 1 on
  PackPool* pack_pool = nullptr;
  std::vector<uint8_t*> hpack;         // ring_depth pinned host slots of ldp x bs bytes
  std::vector<cudaEvent_t> ev_staged;  // the copy out of hpack[slot] has finished
  int64_t h2d_bytes = 0;             // SNP-block bytes copied host -> device
  void* static_scratch = nullptr;  // device address of the fixed scratch array (gwas_solve_block_static)
  int64_t launches = 0;
  int64_t not_spd_index = -1;
  std::string detail;
  // stage timing (measurement only)
  bool timing = false;
  struct Mark { int stage; cudaEvent_t a, b; };
  std::vector<Mark> marks;
  std::vector<cudaEvent_t> event_pool;
};

namespace {

thread_local int64_t tl_init_not_spd = -1;
thread_local std::string tl_init_detail;

int fail(gwas_ctx* c, int code, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->detail = buf;
  }
  return code;
}

#define CK(call)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? GWAS_ERR_NOMEM : GWAS_ERR_CUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                              \
  } while (0)

bool is_device_ptr(const void* ptr) {
  if (!ptr) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <typename T>
cudaError_t dmalloc(T** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return cudaSuccess;
  return cudaMalloc(reinterpret_cast<void**>(p), bytes);
}

cudaEvent_t pool_event(gwas_ctx* c) {
  if (!c->event_pool.empty()) {
    cudaEvent_t e = c->event_pool.back();
    c->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Brackets one stage with events on stream s when timing is on.
struct StageMark {
  gwas_ctx* c;
  int stage;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  StageMark(gwas_ctx* c_, int stage_, cudaStream_t s_) : c(c_), stage(stage_), s(s_) {
    if (c->timing) {
      a = pool_event(c);
      cudaEventRecord(a, s);
    }
  }
  ~StageMark() {
    if (a) {
      cudaEvent_t b = pool_event(c);
      cudaEventRecord(b, s);
      c->marks.push_back({stage, a, b});
    }
  }
};

// Reads the device status block; returns a GWAS code (TIMEOUT) and clears it.
int check_device_status(gwas_ctx* ctx) {
  DevStatus hs;
  CK(cudaMemcpyAsync(&hs, ctx->st, sizeof hs, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (hs.err != DEV_OK || hs.abort) {
    DevStatus clean{};
    clean.not_spd = hs.not_spd;
    clean.sc_err = hs.sc_err;
    CK(cudaMemcpy(ctx->st, &clean, sizeof clean, cudaMemcpyHostToDevice));
    if (hs.err == DEV_ERR_RANGE)
      return fail(ctx, GWAS_ERR_ARG, "SNP values too large for the exact products (largest |x - c| times "
                                     "n_pad times the slice bound, 512 in the adjoint and 1024 in the sliced "
                                     "solve, reaches 2^31)");
    return fail(ctx, GWAS_ERR_TIMEOUT, "a bounded device-side wait ran out (device code %d)", hs.err);
  }
  return GWAS_OK;
}

// out = L^-1 X (upper = false) or L^-T X (upper = true) for FP64 columns, FP64 solve.
// tri_col0 >= 0 (lower): X holds identity columns tri_col0 .. (zero tiles skipped).
int solve_f64_cols(gwas_ctx* ctx, const double* X, int64_t ldx, int rows, int ncols, double* out, bool upper,
                   int64_t tri_col0 = -1) {
  for (int c0 = 0; c0 < ncols; c0 += ctx->bs) {
    const int nc = std::min(ctx->bs, ncols - c0);
    const int C64 = (nc + F64_TN - 1) / F64_TN;
    CK(cudaMemsetAsync(ctx->sched, 0, sizeof(Sched) + sizeof(int) * (size_t)ctx->P * C64, ctx->stream));
    TrsmF64Args a{};
    a.Aop = upper ? ctx->AopT : ctx->Aop; a.lda = ctx->n_pad;
    a.X = X + (int64_t)c0 * ldx; a.ldx = ldx; a.n = rows;
    a.Xt = out + (int64_t)c0 * ctx->n_pad; a.ldt = ctx->n_pad;
    a.P = ctx->P; a.ncols = nc; a.C = C64;
    a.sched = ctx->sched; a.st = ctx->st;
    a.tri_col0 = (tri_col0 >= 0 && !upper) ? tri_col0 + c0 : -1;
    CK(launch_trsm_f64(a, false, ctx->stream, ctx->num_sms, upper));
    ctx->launches += 1;
  }
  return GWAS_OK;
}

// The transpose block operator (for L^-T solves).
int ensure_aop_t(gwas_ctx* ctx) {
  if (ctx->AopT) return GWAS_OK;
  const size_t np = (size_t)ctx->n_pad;
  CK(dmalloc(&ctx->AopT, sizeof(double) * np * np));
  CK(cudaMemsetAsync(ctx->AopT, 0, sizeof(double) * np * np, ctx->stream));
  CK(launch_build_aop_t(ctx->L, ctx->Dinv, ctx->n_pad, ctx->AopT, ctx->stream, &ctx->launches));
  return GWAS_OK;
}

// W = M^-1 = L^-T L^-1 in FP64 (n_pad x n_pad, zero on the padding): the FP64
// solves of the identity, bs columns at a time.  *out receives the device array.
int form_inverse(gwas_ctx* ctx, double** out) {
  *out = nullptr;
  int rc = ensure_aop_t(ctx);
  if (rc != GWAS_OK) return rc;
  const size_t np = (size_t)ctx->n_pad;
  const int n = ctx->n;
  double *W = nullptr, *E = nullptr;
  rc = [&]() -> int {
    CK(dmalloc(&W, sizeof(double) * np * np));
    CK(cudaMemsetAsync(W, 0, sizeof(double) * np * np, ctx->stream));
    CK(dmalloc(&E, sizeof(double) * (size_t)n * std::min(ctx->bs, n)));
    for (int c0 = 0; c0 < n; c0 += ctx->bs) {
      const int ncc = std::min(ctx->bs, n - c0);
      CK(launch_identity_cols(E, n, c0, ncc, ctx->stream));
      ctx->launches += 1;
      int r = solve_f64_cols(ctx, E, n, n, ncc, ctx->Xt, false, c0);
      if (r == GWAS_OK) r = solve_f64_cols(ctx, ctx->Xt, ctx->n_pad, ctx->n_pad, ncc, W + (size_t)c0 * np, true);
      if (r != GWAS_OK) return r;
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return GWAS_OK;
  }();
  cudaFree(E);
  if (rc != GWAS_OK) {
    cudaFree(W);
    return rc;
  }
  *out = W;
  return GWAS_OK;
}

// The adjoint's loop-invariant part: the transpose operator, X^_L and y^, their Gram.
int ensure_adjoint(gwas_ctx* ctx) {
  if (ctx->adjoint_ready) return GWAS_OK;
  const size_t np = (size_t)ctx->n_pad;
  const int nc = ctx->q + 1;
  int rc0 = ensure_aop_t(ctx);
  if (rc0 != GWAS_OK) return rc0;
  // each array once (a failed earlier attempt may have made some of them)
  if (!ctx->Xhat) CK(dmalloc(&ctx->Xhat, sizeof(double) * np * std::max(ctx->bs, nc)));
  if (!ctx->What) CK(dmalloc(&ctx->What, sizeof(double) * np * nc));
  if (!ctx->GH) CK(dmalloc(&ctx->GH, sizeof(double) * nc * nc));
  if (!ctx->adj)
    CK(dmalloc(&ctx->adj, sizeof(double) * ((size_t)ctx->bs * (2 + ctx->p) + QMAX + 1 + ctx->n +
                                             (size_t)adjoint_dy_chunks(ctx->bs) * ctx->n)));
  int rc = solve_f64_cols(ctx, ctx->W, ctx->n_pad, ctx->n_pad, nc, ctx->What, true);
  if (rc != GWAS_OK) return rc;
  CK(launch_gram(ctx->What, ctx->n_pad, ctx->n_pad, nc, ctx->GH, ctx->stream));
  ctx->launches += 1;
  ctx->adjoint_ready = true;
  return GWAS_OK;
}

// The split precisions' adjoint set-up: W = M^-1 (form_inverse), W [X^_L | y^]
// by the FP64 solves, then the exact slices of both (exact_adjoint_create).
int ensure_exact_adjoint(gwas_ctx* ctx) {
  if (ctx->exact) return GWAS_OK;
  int rc = ensure_adjoint(ctx);
  if (rc != GWAS_OK) return rc;
  const size_t np = (size_t)ctx->n_pad;
  const int n = ctx->n, nc = ctx->q + 1;
  double *W = nullptr, *W2 = nullptr;
  auto release = [&] {
    cudaFree(W);
    cudaFree(W2);
  };
  rc = [&]() -> int {
    int r = form_inverse(ctx, &W);
    if (r != GWAS_OK) return r;
    CK(dmalloc(&W2, sizeof(double) * np * nc));
    r = solve_f64_cols(ctx, ctx->What, ctx->n_pad, ctx->n_pad, nc, ctx->Xt, false);
    if (r == GWAS_OK) r = solve_f64_cols(ctx, ctx->Xt, ctx->n_pad, ctx->n_pad, nc, W2, true);
    if (r != GWAS_OK) return r;
    double* Wt = W;
    W = nullptr;  // owned by the exact state from here on, failures included
    CK(exact_adjoint_create(&ctx->exact, Wt, ctx->What, W2, n, ctx->n_pad, ctx->q, ctx->bs, ctx->intercept,
                            ctx->num_sms, ctx->stream, &ctx->launches));
    return check_device_status(ctx);
  }();
  release();
  return rc;
}

// X~ = L^-1 X for one block (FP64 or split precision), then reductions + solve.
// packed: X holds 2-bit packed columns (ldx bytes a column, 16-byte aligned),
// which only the split inverse form reads as they are (tc::packed_ok).
int run_block(gwas_ctx* ctx, const void* X, bool int8_input, int64_t ldx, int ncols, double* b, double* se,
              int* status, bool packed = false) {
  if (packed && !(ctx->tcs && tc::packed_ok(ctx->tcs)))
    return fail(ctx, GWAS_ERR_ARG, "packed columns go to the split inverse form only");
  const int C64 = (ncols + F64_TN - 1) / F64_TN;
  if (ctx->prec == GWAS_FP64 || !int8_input) {
    CK(cudaMemsetAsync(ctx->sched, 0, sizeof(Sched) + sizeof(int) * (size_t)ctx->P * C64, ctx->stream));
    TrsmF64Args a{};
    a.Aop = ctx->Aop; a.lda = ctx->n_pad;
    a.X = X; a.ldx = ldx; a.n = ctx->n;
    a.Xt = ctx->Xt; a.ldt = ctx->n_pad;
    a.P = ctx->P; a.ncols = ncols; a.C = C64;
    a.sched = ctx->sched; a.st = ctx->st;
    {
      StageMark m(ctx, GWAS_STAGE_TRSM, ctx->stream);
      StageMark k(ctx, GWAS_STAGE_SOLVE, ctx->stream);
      CK(launch_trsm_f64(a, int8_input, ctx->stream, ctx->num_sms));
    }
    ctx->launches += 1;
    {
      StageMark m(ctx, GWAS_STAGE_REDUCE, ctx->stream);
      CK(launch_reduce_solve(ctx->Xt, XT_F64, ctx->n_pad, ctx->n_pad, ctx->W, ctx->n_pad, ctx->sc, ctx->q, ncols,
                             b, se, status, ctx->stream, nullptr, nullptr, nullptr, 0, nullptr, ctx->t));
    }
    ctx->launches += 1;
    return GWAS_OK;
  }
  if (ctx->prec == GWAS_SLICED64) {  // exact products of the sliced M^-1 (any alignment of X)
    int64_t nl = 0;
    {
      StageMark m(ctx, GWAS_STAGE_TRSM, ctx->stream);
      cudaEvent_t k0 = ctx->timing ? pool_event(ctx) : nullptr, k1 = ctx->timing ? pool_event(ctx) : nullptr;
      cudaError_t e = exact_solve_product(ctx->sliced, static_cast<const int8_t*>(X), ldx, ncols, ctx->st,
                                          ctx->stream, k0, k1);
      if (ctx->timing && e == cudaSuccess) {
        ctx->marks.push_back({GWAS_STAGE_SOLVE, k0, k1});
      } else if (ctx->timing) {
        ctx->event_pool.push_back(k0);
        ctx->event_pool.push_back(k1);
      }
      if (e != cudaSuccess) return fail(ctx, GWAS_ERR_CUDA, "sliced solve: %s", cudaGetErrorString(e));
      nl += 2;
    }
    {
      StageMark m(ctx, GWAS_STAGE_REDUCE, ctx->stream);
      CK(exact_solve_sums(ctx->sliced, ncols, ctx->sc, ctx->t, b, se, status, ctx->stream));
      nl += 1;
    }
    ctx->launches += nl;
    return GWAS_OK;
  }
  // split precision: the TMA map of X needs a 16-byte aligned base and leading dimension
  const int8_t* X8 = static_cast<const int8_t*>(X);
  if (!packed && ((reinterpret_cast<uintptr_t>(X8) & 15) || (ldx & 15))) {
    CK(cudaMemcpy2DAsync(ctx->ring[0], (size_t)ctx->n_pad, X8, (size_t)ldx, (size_t)ctx->n, (size_t)ncols,
                         cudaMemcpyDeviceToDevice, ctx->stream));
    X8 = ctx->ring[0];
    ldx = ctx->n_pad;
  }
  {
    StageMark m(ctx, GWAS_STAGE_TRSM, ctx->stream);
    int64_t nl = 0;
    cudaEvent_t k0 = ctx->timing ? pool_event(ctx) : nullptr, k1 = ctx->timing ? pool_event(ctx) : nullptr;
    cudaError_t e = tc::run_block(ctx->tcs, X8, ldx, ncols, ctx->stream, &nl, k0, k1, packed);
    if (ctx->timing && e == cudaSuccess) {
      ctx->marks.push_back({GWAS_STAGE_SOLVE, k0, k1});
    } else if (ctx->timing) {
      ctx->event_pool.push_back(k0);
      ctx->event_pool.push_back(k1);
    }
    ctx->launches += nl;
    if (e != cudaSuccess) return fail(ctx, GWAS_ERR_CUDA, "split-precision solve: %s", cudaGetErrorString(e));
  }
  {
    StageMark m(ctx, GWAS_STAGE_REDUCE, ctx->stream);
    if (const float* red = tc::partials(ctx->tcs))  // the sums were formed inside the solve
      CK(launch_partials_solve(red, tc::partial_groups(ctx->tcs), tc::partial_ld(ctx->tcs), ctx->sc, ctx->q, ctx->t,
                               ncols, b, se, status, tc::shift_of(ctx->tcs), ctx->stream));
    else
      CK(launch_reduce_solve(tc::xt_f32(ctx->tcs), XT_F32, tc::xt_ld(ctx->tcs), ctx->n_pad, ctx->W, ctx->n_pad,
                             ctx->sc, ctx->q, ncols, b, se, status, ctx->stream, ctx->W32, tc::shift_of(ctx->tcs),
                             ctx->st, ctx->num_sms, tc::xt_reduce_map(ctx->tcs), ctx->t));
  }
  ctx->launches += 1;
  return GWAS_OK;
}

int solve_common(gwas_ctx* ctx, const void* XR, bool int8_input, int64_t ldx, int ncols, double* b, double* se,
                 int* status) {
  if (!ctx) return GWAS_ERR_ARG;
  if (!XR || !b || ncols < 0 || ncols > ctx->bs || ldx < ctx->n)
    return fail(ctx, GWAS_ERR_ARG, "bad arguments: XR=%p b=%p ncols=%d (bs %d) ldx=%lld (n %d)", XR, (void*)b,
                ncols, ctx->bs, (long long)ldx, ctx->n);
  if (ncols == 0) return GWAS_OK;
  DeviceScope dscope_(ctx->dev);
  CK(dscope_.status());
  const bool dev_in = is_device_ptr(XR);
  const bool dev_out = is_device_ptr(b) && (!se || is_device_ptr(se)) && (!status || is_device_ptr(status));
  const void* xin = XR;
  int64_t ld_in = ldx;
  if (!dev_in) {
    StageMark m(ctx, GWAS_STAGE_H2D, ctx->stream);
    if (int8_input) {
      CK(cudaMemcpy2DAsync(ctx->ring[0], (size_t)ctx->n_pad, XR, (size_t)ldx, (size_t)ctx->n, (size_t)ncols,
                           cudaMemcpyHostToDevice, ctx->stream));
      ctx->h2d_bytes += (int64_t)ctx->n * ncols;
      xin = ctx->ring[0];
      ld_in = ctx->n_pad;
    } else {
      if (!ctx->f64_in) CK(dmalloc(&ctx->f64_in, sizeof(double) * (size_t)ctx->n * ctx->bs));
      CK(cudaMemcpy2DAsync(ctx->f64_in, sizeof(double) * (size_t)ctx->n, XR, sizeof(double) * (size_t)ldx,
                           sizeof(double) * (size_t)ctx->n, (size_t)ncols, cudaMemcpyHostToDevice, ctx->stream));
      ctx->h2d_bytes += (int64_t)sizeof(double) * ctx->n * ncols;
      xin = ctx->f64_in;
      ld_in = ctx->n;
    }
  }
  double* ob = dev_out ? b : ctx->d_b;
  double* ose = dev_out ? se : (se ? ctx->d_se : nullptr);
  int* ost = dev_out ? status : (status ? ctx->d_status : nullptr);
  int rc = run_block(ctx, xin, int8_input, ld_in, ncols, ob, ose, ost);
  if (rc != GWAS_OK) return rc;
  if (dev_in && dev_out) return GWAS_OK;  // asynchronous on the context's stream
  if (!dev_out) {
    StageMark m(ctx, GWAS_STAGE_D2H, ctx->stream);
    CK(cudaMemcpyAsync(b, ctx->d_b, sizeof(double) * (size_t)ctx->p * ncols * ctx->t, cudaMemcpyDeviceToHost,
                       ctx->stream));
    if (se)
      CK(cudaMemcpyAsync(se, ctx->d_se, sizeof(double) * (size_t)ctx->p * ncols, cudaMemcpyDeviceToHost,
                         ctx->stream));
    if (status)
      CK(cudaMemcpyAsync(status, ctx->d_status, sizeof(int) * (size_t)ncols, cudaMemcpyDeviceToHost, ctx->stream));
  }
  return check_device_status(ctx);
}

void free_all(gwas_ctx* c) {
  if (!c) return;
  DeviceScope dscope_(c->dev);
  cudaStreamSynchronize(c->stream);
  if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
  if (c->out_stream) cudaStreamSynchronize(c->out_stream);
  for (auto* p : c->ring) cudaFree(p);
  for (auto& v : {&c->ev_copied, &c->ev_free, &c->ev_out})
    for (auto ev : *v) cudaEventDestroy(ev);
  for (auto& mk : c->marks) { cudaEventDestroy(mk.a); cudaEventDestroy(mk.b); }
  for (auto ev : c->event_pool) cudaEventDestroy(ev);
  cudaFree(c->L); cudaFree(c->Dinv); cudaFree(c->Aop); cudaFree(c->W); cudaFree(c->G);
  cudaFree(c->sc); cudaFree(c->st); cudaFree(c->Xt); cudaFree(c->sched);
  cudaFree(c->d_b); cudaFree(c->d_se); cudaFree(c->d_status); cudaFree(c->f64_in); cudaFree(c->W32);
  cudaFree(c->AopT); cudaFree(c->Xhat); cudaFree(c->What); cudaFree(c->GH); cudaFree(c->adj);
  cudaFreeHost(c->h_b); cudaFreeHost(c->h_se); cudaFreeHost(c->h_status);
  for (auto* p : c->dpack) cudaFree(p);
  for (auto* p : c->hpack) cudaFreeHost(p);
  for (auto ev : c->ev_staged) cudaEventDestroy(ev);
  pack_pool_destroy(c->pack_pool);
  if (c->tcs) tc::destroy(c->tcs);
  exact_destroy(c->exact);
  exact_destroy(c->sliced);
  for (auto* p : c->file_buf) cudaFreeHost(p);
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  if (c->out_stream) cudaStreamDestroy(c->out_stream);
  delete c;
}

}  // namespace

extern "C" {

void gwas_config_default(gwas_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof *cfg);
  cfg->precision = GWAS_FP64;
  cfg->bs = 4096;
  cfg->ring_depth = 3;
  cfg->device = -1;
  cfg->stream_pack = -1;
}

const char* gwas_strerror(int code) {
  switch (code) {
    case GWAS_OK: return "ok";
    case GWAS_ERR_ARG: return "invalid argument";
    case GWAS_ERR_NOT_SPD: return "matrix not positive definite";
    case GWAS_ERR_CUDA: return "CUDA error";
    case GWAS_ERR_TIMEOUT: return "bounded wait timed out";
    case GWAS_ERR_IO: return "input/output error";
    case GWAS_ERR_NOMEM: return "out of memory";
    case GWAS_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown error";
  }
}

const char* gwas_last_error_detail(const gwas_ctx* ctx) { return ctx ? ctx->detail.c_str() : tl_init_detail.c_str(); }

int gwas_init(gwas_ctx** out, int n, int p, const double* phi_or_L, int is_L, const double* XL, const double* y,
              double h, double sigma2, const gwas_config* cfg_in, void* stream) {
  if (!out) return GWAS_ERR_ARG;
  *out = nullptr;
  gwas_config cfg;
  gwas_config_default(&cfg);
  if (cfg_in) cfg = *cfg_in;
  if (n < 1 || p < 1 || p > QMAX + 1 || !phi_or_L || !y || (p > 1 && !XL) || !(h >= 0.0 && h <= 1.0) ||
      !(sigma2 > 0.0) || cfg.bs < 1 || cfg.ring_depth < 2 || cfg.strip_group < 0 || cfg.tile_mode < GWAS_TILES_AUTO || cfg.tile_mode > GWAS_TILES_INVERSE ||
      cfg.tile_mode == 2 /* not a mode */ ||
      cfg.precision < GWAS_FP64 || cfg.precision > GWAS_SLICED64 ||
      (cfg.precision == GWAS_F16X2 && cfg.tile_mode != GWAS_TILES_AUTO && cfg.tile_mode != GWAS_TILES_INVERSE))
    return GWAS_ERR_ARG;
  if (cfg.separate_sums != 0 && cfg.separate_sums != 1) return GWAS_ERR_ARG;
  if (cfg.precision == GWAS_SLICED64 &&
      (cfg.tile_mode != GWAS_TILES_AUTO || cfg.strip_group != 0 || cfg.separate_sums != 0 || cfg.single_piece != 0))
    return GWAS_ERR_ARG;
  if (cfg.single_piece != 0 && cfg.single_piece != 1) return GWAS_ERR_ARG;
  if (cfg.stream_pack < -1 || cfg.stream_pack > 1) return GWAS_ERR_ARG;
  if (cfg.single_piece && (cfg.precision == GWAS_FP64 ||
                           (cfg.tile_mode != GWAS_TILES_AUTO && cfg.tile_mode != GWAS_TILES_INVERSE)))
    return GWAS_ERR_ARG;
  const int traits = cfg.traits == 0 ? 1 : cfg.traits;
  if (traits < 1 || traits > TMAX || p - 1 + traits > QMAX + 1) return GWAS_ERR_ARG;

  gwas_ctx* ctx = new gwas_ctx;
  int dev = cfg.device;
  if (dev < 0) {
    if (cudaGetDevice(&dev) != cudaSuccess) {
      cudaGetLastError();
      free_all(ctx);
      return GWAS_ERR_CUDA;
    }
  }
  ctx->dev = dev;
  DeviceScope dscope_(dev);
  if (dscope_.status() != cudaSuccess) {
    cudaGetLastError();
    free_all(ctx);
    return GWAS_ERR_CUDA;
  }
  int rc = [&]() -> int {
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, dev));
    if (prop.major < 10) return fail(ctx, GWAS_ERR_UNSUPPORTED, "device %s (sm_%d%d) is not a Blackwell part",
                                     prop.name, prop.major, prop.minor);
    ctx->num_sms = prop.multiProcessorCount;
    ctx->stream = static_cast<cudaStream_t>(stream);
    CK(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&ctx->out_stream, cudaStreamNonBlocking));
    ctx->n = n; ctx->p = p; ctx->q = p - 1; ctx->t = traits;
    ctx->n_pad = (n + TB - 1) / TB * TB;
    ctx->P = ctx->n_pad / TB;
    ctx->prec = cfg.precision; ctx->bs = cfg.bs; ctx->ring_depth = cfg.ring_depth;
    ctx->separate_sums = cfg.separate_sums != 0;
    ctx->single_piece = cfg.single_piece != 0;
    ctx->stream_pack = cfg.stream_pack;
    ctx->h = h; ctx->sigma2 = sigma2;
    const size_t np = (size_t)ctx->n_pad, n2 = np * np;
    CK(dmalloc(&ctx->L, sizeof(double) * n2));
    CK(dmalloc(&ctx->Dinv, sizeof(double) * (size_t)ctx->P * TB * TB));
    CK(dmalloc(&ctx->Aop, sizeof(double) * n2));
    const int nw = ctx->q + ctx->t;  // columns of W = [X~_L | Y~]
    CK(dmalloc(&ctx->W, sizeof(double) * np * nw));
    CK(dmalloc(&ctx->G, sizeof(double) * nw * nw));
    CK(dmalloc(&ctx->sc, sizeof(SolveConsts)));
    CK(dmalloc(&ctx->st, sizeof(DevStatus)));
    const int maxC = std::max((cfg.bs + F64_TN - 1) / F64_TN, 1);
    ctx->sched_bytes = sizeof(Sched) + sizeof(int) * (size_t)ctx->P * maxC;
    CK(dmalloc(&ctx->sched, ctx->sched_bytes));
    const int xt_cols = std::max(cfg.bs, nw);
    CK(dmalloc(&ctx->Xt, sizeof(double) * np * xt_cols));
    DevStatus st0{};
    st0.not_spd = ~0ull;
    CK(cudaMemcpyAsync(ctx->st, &st0, sizeof st0, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemsetAsync(ctx->Aop, 0, sizeof(double) * n2, ctx->stream));

    // a1: M (or the given L) into the padded device layout
    const double* src = phi_or_L;
    double* tmp = nullptr;
    if (!is_device_ptr(phi_or_L)) {
      CK(dmalloc(&tmp, sizeof(double) * (size_t)n * n));
      CK(cudaMemcpyAsync(tmp, phi_or_L, sizeof(double) * (size_t)n * n, cudaMemcpyHostToDevice, ctx->stream));
      src = tmp;
    }
    CK(launch_form_m(src, n, n, ctx->n_pad, h, sigma2, is_L, ctx->L, ctx->stream));
    ctx->launches += 1;
    CK(cudaStreamSynchronize(ctx->stream));
    if (tmp) cudaFree(tmp);

    // a2 + a4: Cholesky with the diagonal-block inverses (a given L is refactored
    // from L L^T only in the sense that its diagonal blocks are inverted here)
    double* panel = nullptr;
    CK(dmalloc(&panel, sizeof(double) * np * TB));
    if (!is_L) {
      CK(launch_potrf(ctx->L, ctx->n_pad, ctx->Dinv, panel, ctx->st, ctx->stream, &ctx->launches));
    } else {
      CK(launch_invert_diag_blocks(ctx->L, ctx->n_pad, ctx->Dinv, ctx->st, ctx->stream));
      ctx->launches += 1;
    }
    CK(cudaStreamSynchronize(ctx->stream));
    cudaFree(panel);
    DevStatus hs;
    CK(cudaMemcpy(&hs, ctx->st, sizeof hs, cudaMemcpyDeviceToHost));
    if (hs.not_spd != ~0ull) {
      ctx->not_spd_index = (int64_t)hs.not_spd;
      return fail(ctx, GWAS_ERR_NOT_SPD, "M is not positive definite: pivot %lld", (long long)hs.not_spd);
    }
    CK(launch_build_aop(ctx->L, ctx->Dinv, ctx->n_pad, ctx->Aop, ctx->stream, &ctx->launches));

    // a3: [X~_L | Y~] = L^-1 [X_L | Y] (FP64, t phenotype columns), G = W^T W, solve constants
    double* XLy = nullptr;
    CK(dmalloc(&XLy, sizeof(double) * (size_t)n * nw));
    if (ctx->q) {
      const bool d = is_device_ptr(XL);
      CK(cudaMemcpyAsync(XLy, XL, sizeof(double) * (size_t)n * ctx->q,
                         d ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
    }
    if (ctx->q) {
      std::vector<double> col0(n);
      CK(cudaMemcpyAsync(col0.data(), XLy, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      ctx->intercept = std::all_of(col0.begin(), col0.end(), [](double v) { return v == 1.0; });
    }
    CK(cudaMemcpyAsync(XLy + (size_t)n * ctx->q, y, sizeof(double) * (size_t)n * ctx->t,
                       is_device_ptr(y) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
    {
      const int Cw = (nw + F64_TN - 1) / F64_TN;
      CK(cudaMemsetAsync(ctx->sched, 0, sizeof(Sched) + sizeof(int) * (size_t)ctx->P * Cw, ctx->stream));
      TrsmF64Args a{};
      a.Aop = ctx->Aop; a.lda = ctx->n_pad;
      a.X = XLy; a.ldx = n; a.n = n;
      a.Xt = ctx->W; a.ldt = ctx->n_pad;
      a.P = ctx->P; a.ncols = nw; a.C = Cw;
      a.sched = ctx->sched; a.st = ctx->st;
      CK(launch_trsm_f64(a, false, ctx->stream, ctx->num_sms));
      ctx->launches += 1;
    }
    CK(launch_gram(ctx->W, ctx->n_pad, ctx->n_pad, nw, ctx->G, ctx->stream));
    CK(launch_solve_consts(ctx->G, ctx->q, ctx->t, ctx->sc, ctx->st, ctx->stream));
    ctx->launches += 2;
    CK(cudaStreamSynchronize(ctx->stream));
    cudaFree(XLy);
    CK(cudaMemcpy(&hs, ctx->st, sizeof hs, cudaMemcpyDeviceToHost));
    if (hs.err != DEV_OK) return fail(ctx, GWAS_ERR_TIMEOUT, "set-up solve timed out");
    if (hs.sc_err) return fail(ctx, GWAS_ERR_NOT_SPD, "S_TL = X~_L^T X~_L is singular (collinear covariates)");

    // the sliced solve: W = M^-1, Wh = W [X_L | Y] = L^-T [X~_L | Y~], their slices
    if (ctx->prec == GWAS_SLICED64) {
      int rc0;
      double* Wm = nullptr;
      if ((rc0 = form_inverse(ctx, &Wm)) != GWAS_OK) return rc0;
      double* Wh = nullptr;
      if (dmalloc(&Wh, sizeof(double) * np * nw) != cudaSuccess) {
        cudaFree(Wm);
        return fail(ctx, GWAS_ERR_NOMEM, "sliced set-up: out of device memory");
      }
      rc0 = solve_f64_cols(ctx, ctx->W, ctx->n_pad, ctx->n_pad, nw, Wh, true);
      cudaError_t e = cudaSuccess;
      if (rc0 == GWAS_OK)  // Wm is taken over by the state, on failure too
        e = exact_solve_create(&ctx->sliced, Wm, Wh, nw, ctx->n, ctx->n_pad, ctx->q, cfg.bs, ctx->intercept,
                               ctx->num_sms, ctx->stream, &ctx->launches);
      else
        cudaFree(Wm);
      cudaStreamSynchronize(ctx->stream);
      cudaFree(Wh);
      if (rc0 != GWAS_OK) return rc0;
      if (e != cudaSuccess)
        return fail(ctx, e == cudaErrorMemoryAllocation ? GWAS_ERR_NOMEM : GWAS_ERR_CUDA, "sliced set-up: %s",
                    cudaGetErrorString(e));
      if ((rc0 = check_device_status(ctx)) != GWAS_OK) return rc0;
      cudaFree(ctx->AopT);  // needed again only by the adjoint, which rebuilds it
      ctx->AopT = nullptr;
    }

    // split-precision operands: hi + lo copies of the block operator
    if (ctx->prec != GWAS_FP64 && ctx->prec != GWAS_SLICED64) {
      int64_t nl = 0;
      const tc::Split sp = ctx->prec == GWAS_BF16X3 ? tc::SPLIT_BF16
                           : ctx->prec == GWAS_F16X2 ? tc::SPLIT_F16
                                                     : tc::SPLIT_TF32;
      cudaError_t e = tc::create(&ctx->tcs, sp, ctx->Aop,
                                 ctx->n, ctx->n_pad, cfg.bs, ctx->num_sms, ctx->intercept, ctx->st, ctx->stream,
                                 &nl, cfg.strip_group, static_cast<tc::TileMode>(cfg.tile_mode));
      ctx->launches += nl;
      if (e != cudaSuccess)
        return fail(ctx, e == cudaErrorMemoryAllocation ? GWAS_ERR_NOMEM : GWAS_ERR_CUDA, "split set-up: %s",
                    cudaGetErrorString(e));
      CK(dmalloc(&ctx->W32, sizeof(float) * np * w32_stride(nw - 1)));
      CK(launch_make_w32(ctx->W, ctx->n_pad, ctx->n_pad, nw - 1, ctx->W32, ctx->stream));
      CK(prepare_reduce_solve());
      if (!cfg.separate_sums) CK(tc::set_reductions(ctx->tcs, ctx->W32, w32_stride(nw - 1), nw));
      if (cfg.single_piece) CK(tc::drop_lo_piece(ctx->tcs, ctx->stream));
      ctx->launches += 1;
    }

    // staging: device ring, outputs, pinned result slots, events
    const int R = ctx->ring_depth;
    ctx->ring.assign(R, nullptr);
    for (int i = 0; i < R; ++i) {
      CK(dmalloc(&ctx->ring[i], np * cfg.bs));
      CK(cudaMemsetAsync(ctx->ring[i], 0, np * cfg.bs, ctx->stream));
    }
    CK(dmalloc(&ctx->d_b, sizeof(double) * (size_t)R * p * cfg.bs * ctx->t));
    CK(dmalloc(&ctx->d_se, sizeof(double) * (size_t)R * p * cfg.bs));
    CK(dmalloc(&ctx->d_status, sizeof(int) * (size_t)R * cfg.bs));
    CK(cudaMallocHost(&ctx->h_b, sizeof(double) * (size_t)R * p * cfg.bs * ctx->t));
    CK(cudaMallocHost(&ctx->h_se, sizeof(double) * (size_t)R * p * cfg.bs));
    CK(cudaMallocHost(&ctx->h_status, sizeof(int) * (size_t)R * cfg.bs));
    for (auto* v : {&ctx->ev_copied, &ctx->ev_free, &ctx->ev_out}) {
      v->assign(R, nullptr);
      for (auto& ev : *v) CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    // the no-allocation block solve: its scratch array's address and its kernels, loaded now
    CK(static_scratch_setup(&ctx->static_scratch));
    return GWAS_OK;
  }();
  if (rc != GWAS_OK) {
    // a failed set-up leaves no context: its facts stay readable through a NULL context
    tl_init_not_spd = ctx->not_spd_index;
    tl_init_detail = ctx->detail;
    free_all(ctx);
    return rc;
  }
  tl_init_not_spd = -1;
  tl_init_detail.clear();
  *out = ctx;
  return GWAS_OK;
}

int gwas_solve_block(gwas_ctx* ctx, const int8_t* XR, int64_t ldx, int ncols, double* b, double* se, int* status) {
  return solve_common(ctx, XR, true, ldx, ncols, b, se, status);
}

int gwas_solve_block_f64(gwas_ctx* ctx, const double* XR, int64_t ldx, int ncols, double* b, double* se,
                         int* status) {
  return solve_common(ctx, XR, false, ldx, ncols, b, se, status);
}

}  // extern "C"

// Device slots for 2-bit packed columns (ldp = ceil(n/4) rounded up to 16
// bytes per column), allocated on first use.
static int ensure_packed_slots(gwas_ctx* ctx) {
  if (!ctx->dpack.empty()) return GWAS_OK;
  const int64_t ldp = ((ctx->n + 3) / 4 + 15) / 16 * 16;
  std::vector<uint8_t*> slots(ctx->ring_depth, nullptr);
  for (auto& d : slots) {
    const cudaError_t e = dmalloc(&d, (size_t)ldp * ctx->bs);
    if (e != cudaSuccess) {  // nothing half-made stays behind: a later call retries
      for (auto* q : slots) cudaFree(q);
      return fail(ctx, e == cudaErrorMemoryAllocation ? GWAS_ERR_NOMEM : GWAS_ERR_CUDA,
                  "packed input slots: %s", cudaGetErrorString(e));
    }
  }
  ctx->ldp = ldp;
  ctx->dpack = std::move(slots);
  return GWAS_OK;
}

// The 2-bit transport's host side for int8 columns: pinned slots, their
// events and the packing threads, made on the first packed call (nothing
// half-made stays behind; a later call retries).
static int ensure_host_pack(gwas_ctx* ctx) {
  if (!ctx->hpack.empty()) return GWAS_OK;
  const int R = ctx->ring_depth;
  std::vector<uint8_t*> slots(R, nullptr);
  std::vector<cudaEvent_t> evs(R, nullptr);
  cudaError_t e = cudaSuccess;
  for (int s = 0; s < R && e == cudaSuccess; ++s) {
    e = cudaMallocHost(&slots[s], (size_t)ctx->ldp * ctx->bs);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&evs[s], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    for (auto* q : slots)
      if (q) cudaFreeHost(q);
    for (auto ev : evs)
      if (ev) cudaEventDestroy(ev);
    return fail(ctx, e == cudaErrorMemoryAllocation ? GWAS_ERR_NOMEM : GWAS_ERR_CUDA, "host packing slots: %s",
                cudaGetErrorString(e));
  }
  PackPool* pool = pack_pool_create();
  if (!pool) {
    for (auto* q : slots) cudaFreeHost(q);
    for (auto ev : evs) cudaEventDestroy(ev);
    return fail(ctx, GWAS_ERR_NOMEM, "host packing threads could not be started");
  }
  ctx->hpack = std::move(slots);
  ctx->ev_staged = std::move(evs);
  ctx->pack_pool = pool;
  return GWAS_OK;
}

// The whole-study stream over host columns: int8 (ld = ldx bytes per column)
// or 2-bit packed (ld = bytes per packed column).  Int8 columns cross the link
// as int8, or -- with gwas_config.stream_pack -- block by block as 2-bit codes
// packed by host threads while the GPU solves earlier blocks (a block holding
// any value outside 0..3 goes as int8).  Packed blocks are unpacked on the GPU
// (into the ring slot, or by the split inverse form's cast itself).
static int stream_impl(gwas_ctx* ctx, const void* host, bool packed, int64_t ldx, int64_t m, double* b_host,
                       double* se_host, int* status_host) {
  if (!ctx) return GWAS_ERR_ARG;
  const int64_t nb = ((int64_t)ctx->n + 3) / 4;
  if (!host || !b_host || m < 0 || ldx < (packed ? nb : ctx->n))
    return fail(ctx, GWAS_ERR_ARG, "bad arguments to the whole-study stream");
  if (m == 0) return GWAS_OK;
  DeviceScope dscope_(ctx->dev);
  CK(dscope_.status());
  const int R = ctx->ring_depth, bs = ctx->bs, p = ctx->p, T = ctx->t;
  const int64_t nblk = (m + bs - 1) / bs;
  auto cols_of = [&](int64_t blk) { return (int)std::min<int64_t>(bs, m - blk * bs); };
  // Results of block blk are copied out of pinned slot blk % R once its event fired.
  auto drain = [&](int64_t blk) -> int {
    const int slot = (int)(blk % R), nc = cols_of(blk);
    CK(cudaEventSynchronize(ctx->ev_out[slot]));
    // a slot holds the block's phenotypes one after another (p x nc each);
    // phenotype k's p x m results go to b_host + k p m
    for (int k = 0; k < T; ++k)
      std::memcpy(b_host + (k * m + blk * bs) * p, ctx->h_b + (size_t)slot * T * p * bs + (size_t)k * p * nc,
                  sizeof(double) * (size_t)p * nc);
    if (se_host)
      std::memcpy(se_host + blk * bs * p, ctx->h_se + (size_t)slot * p * bs, sizeof(double) * (size_t)p * nc);
    if (status_host)
      std::memcpy(status_host + blk * bs, ctx->h_status + (size_t)slot * bs, sizeof(int) * (size_t)nc);
    return GWAS_OK;
  };
  const uint8_t* src0 = static_cast<const uint8_t*>(host);
  // auto: where the host packs with AVX-512 and the solve outruns the int8
  // link (BF16 / FP16 pieces in the inverse form, whose cast reads the codes)
  const bool outruns_link = ctx->tcs && tc::packed_ok(ctx->tcs) &&
                            (ctx->prec == GWAS_BF16X3 || ctx->prec == GWAS_F16X2);
  const bool host_pack =
      !packed && (ctx->stream_pack == 1 || (ctx->stream_pack == -1 && host_pack_fast() && outruns_link));
  if (packed || host_pack) {
    const int rc0 = ensure_packed_slots(ctx);
    if (rc0 != GWAS_OK) return rc0;
  }
  if (host_pack) {
    const int rc0 = ensure_host_pack(ctx);
    if (rc0 != GWAS_OK) return rc0;
  }
  // Int8 columns whose stride is a multiple of 16 bytes and fits a ring slot
  // are copied as they lie in host memory, one contiguous copy per block (a
  // DMA of whole rows runs a few per cent faster than a pitched one); else the
  // columns are repacked to the slot's stride by a pitched copy.  Packed
  // columns likewise into a slot of ldp bytes per column.
  const int64_t slot_ld_in = packed ? ctx->ldp : ctx->n_pad;
  // the split inverse form's cast reads packed columns themselves (no unpack kernel)
  const bool fused_ok = ctx->tcs && tc::packed_ok(ctx->tcs);
  const int64_t width = packed ? nb : ctx->n;
  const bool flat = (ldx % 16) == 0 && ldx <= slot_ld_in;
  const int64_t ld_dev = flat ? ldx : slot_ld_in;  // the block's leading dimension on the device
  std::vector<char> pk(R, packed ? 1 : 0);          // the block in slot s crossed the link as 2-bit codes
  std::vector<int64_t> ld_slot(R, ld_dev);          // and its leading dimension in its device slot
  auto enqueue_copy = [&](int64_t blk) -> int {
    const int slot = (int)(blk % R), nc = cols_of(blk);
    const uint8_t* src = src0 + blk * bs * ldx;
    bool hp = false;
    if (host_pack) {
      // hpack[slot] last left for the device R blocks ago; packed while the GPU solves earlier blocks
      CK(cudaEventSynchronize(ctx->ev_staged[slot]));
      hp = pack_pool_run(ctx->pack_pool, reinterpret_cast<const int8_t*>(src), ldx, ctx->n, nc, ctx->hpack[slot],
                         ctx->ldp);
    }
    CK(cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_free[slot], 0));
    StageMark mk(ctx, GWAS_STAGE_H2D, ctx->copy_stream);
    if (hp) {
      CK(cudaMemcpyAsync(ctx->dpack[slot], ctx->hpack[slot], (size_t)(ctx->ldp * nc), cudaMemcpyHostToDevice,
                         ctx->copy_stream));
      CK(cudaEventRecord(ctx->ev_staged[slot], ctx->copy_stream));
      ctx->h2d_bytes += ctx->ldp * nc;
      ld_slot[slot] = ctx->ldp;
    } else {
      void* dst = packed ? static_cast<void*>(ctx->dpack[slot]) : static_cast<void*>(ctx->ring[slot]);
      if (flat) {  // the last column ends after its width-th byte
        CK(cudaMemcpyAsync(dst, src, (size_t)((nc - 1) * ldx + width), cudaMemcpyHostToDevice, ctx->copy_stream));
        ctx->h2d_bytes += (nc - 1) * ldx + width;
      } else {
        CK(cudaMemcpy2DAsync(dst, (size_t)slot_ld_in, src, (size_t)ldx, (size_t)width, (size_t)nc,
                             cudaMemcpyHostToDevice, ctx->copy_stream));
        ctx->h2d_bytes += width * nc;
      }
      ld_slot[slot] = ld_dev;
    }
    pk[slot] = packed || hp;
    CK(cudaEventRecord(ctx->ev_copied[slot], ctx->copy_stream));
    return GWAS_OK;
  };
  // the ring starts free
  for (int s = 0; s < R; ++s) CK(cudaEventRecord(ctx->ev_free[s], ctx->stream));
  int rc;
  int64_t next_copy = 0;
  // copies ahead of the first solve: the whole ring, or -- when the host packs
  // each block first -- one block, so that the GPU starts after one packing
  for (; next_copy < std::min<int64_t>(host_pack ? 1 : R, nblk); ++next_copy)
    if ((rc = enqueue_copy(next_copy)) != GWAS_OK) return rc;
  for (int64_t blk = 0; blk < nblk; ++blk) {
    const int slot = (int)(blk % R), nc = cols_of(blk);
    CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_copied[slot], 0));
    const bool fused = pk[slot] && fused_ok;
    if (pk[slot] && !fused) {  // the 2-bit codes into the ring slot as int8
      StageMark mk(ctx, GWAS_STAGE_H2D, ctx->stream);
      CK(launch_unpack2(ctx->dpack[slot], ld_slot[slot], ctx->n, nc, ctx->ring[slot], ctx->n_pad, ctx->stream));
      ctx->launches += 1;
    }
    double* ob = ctx->d_b + (size_t)slot * T * p * bs;
    double* ose = ctx->d_se + (size_t)slot * p * bs;
    int* ost = ctx->d_status + (size_t)slot * bs;
    // the slot's outputs were copied out R blocks ago (on the result stream)
    if (blk >= R) CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_out[slot], 0));
    rc = fused ? run_block(ctx, ctx->dpack[slot], true, ld_slot[slot], nc, ob, ose, ost, true)
               : run_block(ctx, ctx->ring[slot], true, pk[slot] ? ctx->n_pad : ld_slot[slot], nc, ob, ose, ost);
    if (rc != GWAS_OK) return rc;
    CK(cudaEventRecord(ctx->ev_free[slot], ctx->stream));
    {  // results out on their own stream, overlapping the next block's solve
    CK(cudaStreamWaitEvent(ctx->out_stream, ctx->ev_free[slot], 0));
    StageMark mk(ctx, GWAS_STAGE_D2H, ctx->out_stream);
    CK(cudaMemcpyAsync(ctx->h_b + (size_t)slot * T * p * bs, ob, sizeof(double) * (size_t)p * nc * T,
                       cudaMemcpyDeviceToHost, ctx->out_stream));
    if (se_host)
      CK(cudaMemcpyAsync(ctx->h_se + (size_t)slot * p * bs, ose, sizeof(double) * (size_t)p * nc,
                         cudaMemcpyDeviceToHost, ctx->out_stream));
    if (status_host)
      CK(cudaMemcpyAsync(ctx->h_status + (size_t)slot * bs, ost, sizeof(int) * (size_t)nc,
                         cudaMemcpyDeviceToHost, ctx->out_stream));
    }
    CK(cudaEventRecord(ctx->ev_out[slot], ctx->out_stream));
    for (; next_copy < nblk && next_copy <= blk + R; ++next_copy)  // the ring refilled up to R blocks ahead
      if ((rc = enqueue_copy(next_copy)) != GWAS_OK) return rc;
    // results of the previous block: its copy-out overlaps this block's solve
    if (blk >= 1 && (rc = drain(blk - 1)) != GWAS_OK) return rc;
  }
  if ((rc = drain(nblk - 1)) != GWAS_OK) return rc;
  return check_device_status(ctx);
}

extern "C" {

int gwas_solve_stream(gwas_ctx* ctx, const int8_t* XR_host, int64_t ldx, int64_t m, double* b_host,
                      double* se_host, int* status_host) {
  return stream_impl(ctx, XR_host, false, ldx, m, b_host, se_host, status_host);
}

int gwas_solve_stream_packed(gwas_ctx* ctx, const uint8_t* P_host, int64_t ldp, int64_t m, double* b_host,
                             double* se_host, int* status_host) {
  return stream_impl(ctx, P_host, true, ldp, m, b_host, se_host, status_host);
}

}  // extern "C"

// Disk -> pinned host -> GPU over columns col0 .. col0+m-1 of a file; `sink`
// receives each block's results (pinned host slices of b, se, status) in
// column order, while the GPU works on later blocks.
template <typename Sink>
static int solve_file_impl(gwas_ctx* ctx, const char* path, int64_t header_bytes, int64_t ldx, int64_t col0, int64_t m,
                           bool packed, bool want_se, bool want_status, Sink&& sink) {
  DeviceScope dscope_(ctx->dev);
  CK(dscope_.status());
  const int R = ctx->ring_depth, bs = ctx->bs, p = ctx->p;
  // packed columns (2-bit codes, ceil(n/4) bytes) land in a device slot of
  // ldp bytes per column and are unpacked into the ring slot
  const int64_t width = packed ? ((int64_t)ctx->n + 3) / 4 : ctx->n;
  const bool fused = packed && ctx->tcs && tc::packed_ok(ctx->tcs);  // the cast reads the packed columns
  if (packed) {
    const int r0 = ensure_packed_slots(ctx);
    if (r0 != GWAS_OK) return r0;
  }
  const int64_t nblk = (m + bs - 1) / bs;
  auto cols_of = [&](int64_t blk) { return (int)std::min<int64_t>(bs, m - blk * bs); };
  if (ctx->file_buf_bytes < ldx * bs) {
    for (auto* q : ctx->file_buf) cudaFreeHost(q);
    ctx->file_buf.assign(3, nullptr);
    ctx->file_buf_bytes = 0;
    for (auto& q : ctx->file_buf) CK(cudaMallocHost(&q, (size_t)(ldx * bs)));
    ctx->file_buf_bytes = ldx * bs;
  }
  gwas_reader* rd = nullptr;
  int rc = reader_open_with(&rd, path, header_bytes + col0 * ldx, ldx * bs, nblk, ldx * cols_of(nblk - 1), 3,
                            ctx->file_buf.data());
  if (rc != GWAS_OK) return fail(ctx, rc, "cannot open %s", path);
  auto drain = [&](int64_t blk) -> int {
    const int slot = (int)(blk % R);
    CK(cudaEventSynchronize(ctx->ev_out[slot]));
    return sink(blk, cols_of(blk), ctx->h_b + (size_t)slot * ctx->t * p * bs, ctx->h_se + (size_t)slot * p * bs,
                ctx->h_status + (size_t)slot * bs);
  };
  rc = [&]() -> int {
    for (int sl = 0; sl < R; ++sl) CK(cudaEventRecord(ctx->ev_free[sl], ctx->stream));
    for (int64_t blk = 0; blk < nblk; ++blk) {
      const int slot = (int)(blk % R), nc = cols_of(blk);
      const void* hb = nullptr;
      int64_t got = 0;
      int r2 = gwas_reader_next(rd, &hb, &got, 120000);
      if (r2 != GWAS_OK) return fail(ctx, r2, "reading block %lld: %s", (long long)blk, gwas_reader_error_detail(rd));
      CK(cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_free[slot], 0));
      {
        StageMark mk(ctx, GWAS_STAGE_H2D, ctx->copy_stream);
        if (packed)
          CK(cudaMemcpy2DAsync(ctx->dpack[slot], (size_t)ctx->ldp, hb, (size_t)ldx, (size_t)width, (size_t)nc,
                               cudaMemcpyHostToDevice, ctx->copy_stream));
        else
          CK(cudaMemcpy2DAsync(ctx->ring[slot], (size_t)ctx->n_pad, hb, (size_t)ldx, (size_t)ctx->n, (size_t)nc,
                               cudaMemcpyHostToDevice, ctx->copy_stream));
        ctx->h2d_bytes += width * nc;
      }
      CK(cudaEventRecord(ctx->ev_copied[slot], ctx->copy_stream));
      CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_copied[slot], 0));
      if (packed && !fused) {
        StageMark mk(ctx, GWAS_STAGE_H2D, ctx->stream);
        CK(launch_unpack2(ctx->dpack[slot], ctx->ldp, ctx->n, nc, ctx->ring[slot], ctx->n_pad, ctx->stream));
        ctx->launches += 1;
      }
      double* ob = ctx->d_b + (size_t)slot * ctx->t * p * bs;
      double* ose = ctx->d_se + (size_t)slot * p * bs;
      int* ost = ctx->d_status + (size_t)slot * bs;
      r2 = fused ? run_block(ctx, ctx->dpack[slot], true, ctx->ldp, nc, ob, ose, ost, true)
                 : run_block(ctx, ctx->ring[slot], true, ctx->n_pad, nc, ob, ose, ost);
      if (r2 != GWAS_OK) return r2;
      CK(cudaEventRecord(ctx->ev_free[slot], ctx->stream));
      {
        StageMark mk(ctx, GWAS_STAGE_D2H, ctx->stream);
        CK(cudaMemcpyAsync(ctx->h_b + (size_t)slot * ctx->t * p * bs, ob, sizeof(double) * (size_t)p * nc * ctx->t,
                           cudaMemcpyDeviceToHost, ctx->stream));
        if (want_se)
          CK(cudaMemcpyAsync(ctx->h_se + (size_t)slot * p * bs, ose, sizeof(double) * (size_t)p * nc,
                             cudaMemcpyDeviceToHost, ctx->stream));
        if (want_status)
          CK(cudaMemcpyAsync(ctx->h_status + (size_t)slot * bs, ost, sizeof(int) * (size_t)nc, cudaMemcpyDeviceToHost,
                             ctx->stream));
      }
      CK(cudaEventRecord(ctx->ev_out[slot], ctx->stream));
      // the host buffer of the previous block goes back to the reader once its copy landed
      if (blk >= 1) {
        CK(cudaEventSynchronize(ctx->ev_copied[(blk - 1) % R]));
        gwas_reader_release(rd);
        if ((r2 = drain(blk - 1)) != GWAS_OK) return r2;
      }
    }
    CK(cudaEventSynchronize(ctx->ev_copied[(nblk - 1) % R]));
    gwas_reader_release(rd);
    int r3 = drain(nblk - 1);
    if (r3 != GWAS_OK) return r3;
    return check_device_status(ctx);
  }();
  gwas_reader_close(rd);
  return rc;
}

// ------------------------------------------------ disk to disk, resumable
namespace {
struct ResHeader {  // the result file's and the checkpoint's first 64 bytes
  char magic[8];
  uint32_t version, p;
  uint64_t n, col0, m;
  uint32_t record_bytes, precision;
  uint64_t done;    // checkpoint only: columns whose records are on disk
  uint64_t traits;  // phenotypes per record
};
static_assert(sizeof(ResHeader) == 64, "64-byte header");

bool write_all(int fd, const void* buf, size_t bytes, int64_t off) {
  const char* p = static_cast<const char*>(buf);
  while (bytes > 0) {
    const ssize_t w = pwrite(fd, p, bytes, (off_t)off);
    if (w < 0 && errno == EINTR) continue;
    if (w <= 0) return false;
    p += w;
    bytes -= (size_t)w;
    off += w;
  }
  return true;
}

bool read_all(int fd, void* buf, size_t bytes, int64_t off) {
  char* p = static_cast<char*>(buf);
  while (bytes > 0) {
    const ssize_t r = pread(fd, p, bytes, (off_t)off);
    if (r < 0 && errno == EINTR) continue;
    if (r <= 0) return false;
    p += r;
    bytes -= (size_t)r;
    off += r;
  }
  return true;
}
}  // namespace

extern "C" {

int gwas_solve_file(gwas_ctx* ctx, const char* path, int64_t header_bytes, int64_t ldx, int64_t col0, int64_t m,
                    double* b_host, double* se_host, int* status_host) {
  if (!ctx) return GWAS_ERR_ARG;
  if (!path || !b_host || header_bytes < 0 || ldx < ctx->n || col0 < 0 || m < 0)
    return fail(ctx, GWAS_ERR_ARG, "bad arguments to gwas_solve_file");
  if (m == 0) return GWAS_OK;
  const int p = ctx->p, bs = ctx->bs;
  return solve_file_impl(ctx, path, header_bytes, ldx, col0, m, false, se_host != nullptr, status_host != nullptr,
                         [&](int64_t blk, int nc, const double* hb, const double* hse, const int* hst) -> int {
                           for (int k = 0; k < ctx->t; ++k)  // phenotype k: p x nc at hb + k p nc
                             std::memcpy(b_host + (k * m + blk * bs) * p, hb + (size_t)k * p * nc,
                                         sizeof(double) * (size_t)p * nc);
                           if (se_host) std::memcpy(se_host + blk * bs * p, hse, sizeof(double) * (size_t)p * nc);
                           if (status_host) std::memcpy(status_host + blk * bs, hst, sizeof(int) * (size_t)nc);
                           return GWAS_OK;
                         });
}

int gwas_solve_file_out(gwas_ctx* ctx, const char* in_path, int64_t header_bytes, int64_t ldx, int64_t col0,
                        int64_t m, const char* out_path, int flags, int64_t* done_out) {
  if (!ctx) return GWAS_ERR_ARG;
  const bool packed_in = (flags & GWAS_PACKED_INPUT) != 0;
  if (!in_path || !out_path || header_bytes < 0 || ldx < (packed_in ? ((int64_t)ctx->n + 3) / 4 : ctx->n) ||
      col0 < 0 || m < 0 || (flags & ~(GWAS_RESUME | GWAS_PACKED_INPUT)))
    return fail(ctx, GWAS_ERR_ARG, "bad arguments to gwas_solve_file_out");
  const int p = ctx->p, bs = ctx->bs, T = ctx->t;
  const size_t rec = GWAS_RESULT_RECORD_BYTES_T(p, T);
  ResHeader h{};
  std::memcpy(h.magic, "GWASRES", 8);
  h.version = 1;
  h.p = (uint32_t)p;
  h.n = (uint64_t)ctx->n;
  h.col0 = (uint64_t)col0;
  h.m = (uint64_t)m;
  h.record_bytes = (uint32_t)rec;
  h.precision = (uint32_t)ctx->prec;
  h.traits = (uint64_t)T;
  const std::string ckpt_path = std::string(out_path) + ".ckpt";
  int64_t done = 0;
  const bool resume = (flags & GWAS_RESUME) != 0;
  if (resume) {  // the checkpoint must describe this same run
    const int cfd = open(ckpt_path.c_str(), O_RDONLY);
    if (cfd >= 0) {
      ResHeader c{};
      const bool ok = read_all(cfd, &c, sizeof c, 0);
      close(cfd);
      if (!ok || std::memcmp(c.magic, "GWASCKP", 8) != 0 || c.p != h.p || c.n != h.n || c.col0 != h.col0 ||
          c.m != h.m || c.record_bytes != h.record_bytes || c.precision != h.precision || c.traits != h.traits ||
          c.done > h.m)
        return fail(ctx, GWAS_ERR_ARG, "checkpoint %s does not match this run", ckpt_path.c_str());
      done = (int64_t)c.done;
    }
  }
  const int ofd = open(out_path, O_RDWR | O_CREAT | (resume ? 0 : O_TRUNC), 0644);
  if (ofd < 0) return fail(ctx, GWAS_ERR_IO, "cannot open %s: %s", out_path, strerror(errno));
  const int cfd = open(ckpt_path.c_str(), O_RDWR | O_CREAT, 0644);
  if (cfd < 0) {
    close(ofd);
    return fail(ctx, GWAS_ERR_IO, "cannot open %s: %s", ckpt_path.c_str(), strerror(errno));
  }
  ResHeader ck = h;
  std::memcpy(ck.magic, "GWASCKP", 8);
  // the checkpoint advances only after the records it covers are on disk
  auto checkpoint = [&](int64_t d) -> bool {
    if (fdatasync(ofd) != 0) return false;
    ck.done = (uint64_t)d;
    return write_all(cfd, &ck, sizeof ck, 0) && fdatasync(cfd) == 0;
  };
  int rc = GWAS_OK;
  if (!write_all(ofd, &h, sizeof h, 0) || !checkpoint(done))
    rc = fail(ctx, GWAS_ERR_IO, "writing %s: %s", out_path, strerror(errno));
  if (rc == GWAS_OK && done < m) {
    std::vector<char> buf((size_t)bs * rec);
    const int64_t start = done;
    int64_t since_sync = 0;
    rc = solve_file_impl(ctx, in_path, header_bytes, ldx, col0 + start, m - start, packed_in, true, true,
                         [&](int64_t blk, int nc, const double* hb, const double* hse, const int* hst) -> int {
                           for (int c = 0; c < nc; ++c) {
                             char* r = buf.data() + (size_t)c * rec;
                             for (int k = 0; k < T; ++k)  // phenotype k's block: p x nc at hb + k p nc
                               std::memcpy(r + 8 * p * k, hb + (size_t)k * p * nc + (size_t)c * p,
                                           sizeof(double) * p);
                             std::memcpy(r + 8 * p * T, hse + (size_t)c * p, sizeof(double) * p);
                             const int32_t st[2] = {hst[c], 0};
                             std::memcpy(r + 8 * p * (T + 1), st, 8);
                           }
                           const int64_t first = start + blk * bs;
                           if (!write_all(ofd, buf.data(), (size_t)nc * rec, (int64_t)sizeof h + first * (int64_t)rec))
                             return fail(ctx, GWAS_ERR_IO, "writing %s: %s", out_path, strerror(errno));
                           done = first + nc;
                           // a checkpoint every 16 blocks (and at the end): at most that much is redone
                           if (++since_sync >= 16 || done == m) {
                             since_sync = 0;
                             if (!checkpoint(done))
                               return fail(ctx, GWAS_ERR_IO, "checkpointing %s: %s", ckpt_path.c_str(),
                                           strerror(errno));
                           }
                           return GWAS_OK;
                         });
  }
  close(ofd);
  close(cfd);
  if (done_out) *done_out = done;
  return rc;
}

int gwas_adjoint_block(gwas_ctx* ctx, const int8_t* XR, int64_t ldx, int ncols, double* chi2, double* dchi2_dh,
                       double* dh_accum, double* dy_accum) {
  if (!ctx) return GWAS_ERR_ARG;
  if (!XR || !dh_accum || !dy_accum || ncols < 0 || ncols > ctx->bs || ldx < ctx->n)
    return fail(ctx, GWAS_ERR_ARG, "bad arguments to gwas_adjoint_block");
  if (!(ctx->h > 0.0)) return fail(ctx, GWAS_ERR_ARG, "the adjoint needs h > 0");
  if (ctx->t != 1) return fail(ctx, GWAS_ERR_UNSUPPORTED, "the adjoint takes one phenotype");
  if (ncols == 0) return GWAS_OK;
  DeviceScope dscope_(ctx->dev);
  CK(dscope_.status());
  int rc = ensure_adjoint(ctx);
  if (rc != GWAS_OK) return rc;
  const int p = ctx->p, bs = ctx->bs, n = ctx->n;
  double* d_chi2 = ctx->adj;
  double* d_dh = d_chi2 + bs;
  double* d_w = d_dh + bs;
  double* d_uT = d_w + (size_t)bs * p;
  double* d_acc = d_uT + QMAX;  // [dh, dy...] staging for host accumulators
  double* d_dypart = d_acc + 1 + n;  // the y-gradient's per-chunk partial sums
  const bool dev_acc = is_device_ptr(dh_accum) && is_device_ptr(dy_accum);
  double* acc_dh = dev_acc ? dh_accum : d_acc;
  double* acc_dy = dev_acc ? dy_accum : d_acc + 1;
  if (!dev_acc) {
    CK(cudaMemcpyAsync(d_acc, dh_accum, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(d_acc + 1, dy_accum, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
  }
  // forward solve X~ of the int8 block
  const void* xin = XR;
  int64_t ld_in = ldx;
  const bool split = ctx->prec != GWAS_FP64;
  if (!is_device_ptr(XR) || (split && ((reinterpret_cast<uintptr_t>(XR) & 15) || (ldx & 15)))) {
    CK(cudaMemcpy2DAsync(ctx->ring[0], (size_t)ctx->n_pad, XR, (size_t)ldx, (size_t)n, (size_t)ncols,
                         cudaMemcpyDefault, ctx->stream));
    xin = ctx->ring[0];
    ld_in = ctx->n_pad;
  }
  if (split) {
    // the split adjoint: every per-SNP input from one exact integer product
    // of the sliced [W ; X^_L^T ; y^T ; (W X^_L)^T ; (W y^)^T] with the block's
    // shifted dosages on the tensor cores (exact_products.cu); the per-SNP
    // adjoint arithmetic and the y-gradient in FP64
    if ((rc = ensure_exact_adjoint(ctx)) != GWAS_OK) return rc;
    int64_t nl = 0;
    cudaError_t e;
    {
      StageMark m(ctx, GWAS_STAGE_TRSM, ctx->stream);
      e = exact_adjoint_block(ctx->exact, static_cast<const int8_t*>(xin), ld_in, ncols, ctx->sc, ctx->GH, ctx->What,
                              ctx->h, ctx->sigma2, d_chi2, d_dh, d_w, d_uT, acc_dh, acc_dy, ctx->st, ctx->stream, &nl);
    }
    ctx->launches += nl;
    if (e != cudaSuccess) return fail(ctx, GWAS_ERR_CUDA, "split adjoint: %s", cudaGetErrorString(e));
  } else {
    const int C64 = (ncols + F64_TN - 1) / F64_TN;
    CK(cudaMemsetAsync(ctx->sched, 0, sizeof(Sched) + sizeof(int) * (size_t)ctx->P * C64, ctx->stream));
    TrsmF64Args a{};
    a.Aop = ctx->Aop; a.lda = ctx->n_pad;
    a.X = xin; a.ldx = ld_in; a.n = n;
    a.Xt = ctx->Xt; a.ldt = ctx->n_pad;
    a.P = ctx->P; a.ncols = ncols; a.C = C64;
    a.sched = ctx->sched; a.st = ctx->st;
    StageMark m(ctx, GWAS_STAGE_TRSM, ctx->stream);
    CK(launch_trsm_f64(a, true, ctx->stream, ctx->num_sms));
    ctx->launches += 1;
  }
  // transpose solve X^ = L^-T X~
  if (!split) {
    StageMark m(ctx, GWAS_STAGE_TRSM, ctx->stream);
    if ((rc = solve_f64_cols(ctx, ctx->Xt, ctx->n_pad, ctx->n_pad, ncols, ctx->Xhat, true)) != GWAS_OK) return rc;
  }
  if (!split) {
    StageMark m(ctx, GWAS_STAGE_REDUCE, ctx->stream);
    CK(launch_adjoint(ctx->Xt, ctx->Xhat, ctx->n_pad, ctx->n_pad, n, ctx->W, ctx->What, ctx->n_pad, ctx->sc, ctx->GH,
                      ctx->q, ncols, ctx->h, ctx->sigma2, d_chi2, d_dh, d_w, d_uT, acc_dh, acc_dy, d_dypart,
                      ctx->stream));
    ctx->launches += 4;
  }
  if (chi2)
    CK(cudaMemcpyAsync(chi2, d_chi2, sizeof(double) * ncols, cudaMemcpyDefault, ctx->stream));
  if (dchi2_dh)
    CK(cudaMemcpyAsync(dchi2_dh, d_dh, sizeof(double) * ncols, cudaMemcpyDefault, ctx->stream));
  if (!dev_acc) {
    CK(cudaMemcpyAsync(dh_accum, d_acc, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(dy_accum, d_acc + 1, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
  }
  if (dev_acc && is_device_ptr(XR) && (!chi2 || is_device_ptr(chi2)) && (!dchi2_dh || is_device_ptr(dchi2_dh)))
    return GWAS_OK;
  return check_device_status(ctx);
}

// REML of the null model at one h (FP64 throughout); see gwas_b300.h.
static int reml_eval_impl(const double* phi, int n, int q, const double* XL, const double* y, double h,
                          const gwas_config* cfg, void* stream, double* out) {
  gwas_ctx* ctx = nullptr;
  gwas_config c;
  gwas_config_default(&c);
  if (cfg) c = *cfg;
  c.precision = GWAS_FP64;
  c.bs = std::max(c.bs, q + 1 + 64);  // room for [r~ | X~_L] plus identity chunks in the scratch
  int rc = gwas_init(&ctx, n, q + 1, phi, 0, XL, y, h, 1.0, &c, stream);
  if (rc != GWAS_OK) return rc;
  rc = [&]() -> int {
    DeviceScope dscope_(ctx->dev);
    CK(dscope_.status());
    rc = ensure_adjoint(ctx);
    if (rc != GWAS_OK) return rc;
    const int nc = q + 1, np = ctx->n_pad;
    double* U = ctx->Xt;       // [r~ | X~_L]
    double* Uh = ctx->Xhat;    // [P y | X^_L]  (P y = V^-1 (y - X_L beta) = L^-T r~)
    double* d = ctx->adj;      // scalars
    CK(launch_null_residual(ctx->W, np, np, q, ctx->sc, U, ctx->stream));
    if (q) CK(cudaMemcpyAsync(U + np, ctx->W, sizeof(double) * (size_t)np * q, cudaMemcpyDeviceToDevice, ctx->stream));
    if ((rc = solve_f64_cols(ctx, U, np, np, nc, Uh, true)) != GWAS_OK) return rc;
    CK(launch_log_diag(ctx->L, np, n, d, ctx->stream));                  // d[0] = sum log L_ii
    CK(launch_col_sumsq(U, np, n, 1, d + 1, ctx->stream));               // d[1] = y^T P y
    CK(launch_col_sumsq(Uh, np, n, 1, d + 2, ctx->stream));              // d[2] = ||P y||^2
    if (q) CK(launch_gram(Uh + np, np, np, q, d + 3, ctx->stream));     // d[3..] = X^_L^T X^_L (q x q)
    ctx->launches += 5;
    // tr(V^-1) = ||L^-1||_F^2, columns of the identity in chunks
    double* E = ctx->Xhat + (size_t)np * nc;  // free space after Uh
    const int chunk = std::max(1, std::min(ctx->bs - nc, n));
    double trv = 0.0;
    std::vector<double> part(chunk);
    double* dpart = d + 3 + q * q;
    for (int c0 = 0; c0 < n; c0 += chunk) {
      const int ncc = std::min(chunk, n - c0);
      CK(launch_identity_cols(E, n, c0, ncc, ctx->stream));
      if ((rc = solve_f64_cols(ctx, E, n, n, ncc, ctx->Xt, false)) != GWAS_OK) return rc;
      CK(launch_col_sumsq(ctx->Xt, np, np, ncc, dpart, ctx->stream));
      ctx->launches += 2;
      CK(cudaMemcpyAsync(part.data(), dpart, sizeof(double) * ncc, cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      for (int i = 0; i < ncc; ++i) trv += part[i];
    }
    std::vector<double> hd(3 + q * q);
    SolveConsts hsc;
    CK(cudaMemcpyAsync(hd.data(), d, sizeof(double) * hd.size(), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(&hsc, ctx->sc, sizeof hsc, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if ((rc = check_device_status(ctx)) != GWAS_OK) return rc;
    // A^-1 = Cinv^T Cinv;  log|A| = -2 sum log Cinv_ii;  tr(A^-1 T_LL)
    double logdetA = 0.0, trAT = 0.0;
    for (int i = 0; i < q; ++i) logdetA -= 2.0 * std::log(hsc.Cinv[i + i * QMAX]);
    for (int i = 0; i < q; ++i)
      for (int j = 0; j < q; ++j) {
        double aij = 0.0;
        for (int t = std::max(i, j); t < q; ++t) aij += hsc.Cinv[t + i * QMAX] * hsc.Cinv[t + j * QMAX];
        trAT += aij * hd[3 + j + i * q];
      }
    const double logdetV = 2.0 * hd[0], yPy = hd[1], Py2 = hd[2];
    const double s2 = yPy / (double)(n - q);
    const double trP = trv - trAT;
    out[0] = -0.5 * ((double)(n - q) * std::log(s2) + logdetV + logdetA);
    out[1] = (h > 0.0) ? (trP - Py2 / s2) / (2.0 * h) : std::nan("");
    out[2] = s2;
    return GWAS_OK;
  }();
  if (rc != GWAS_OK) {
    tl_init_detail = ctx->detail;
  }
  gwas_destroy(ctx);
  return rc;
}

int gwas_reml_eval(int n, int q, const double* phi, const double* XL, const double* y, double h,
                   const gwas_config* cfg, void* stream, double* out) {
  if (n < 2 || q < 0 || q >= n || !phi || !y || (q && !XL) || !out || !(h > 0.0 && h <= 1.0)) return GWAS_ERR_ARG;
  return reml_eval_impl(phi, n, q, XL, y, h, cfg, stream, out);
}

int gwas_reml_fit(int n, int q, const double* phi, const double* XL, const double* y, double h0, double tol,
                  int max_evals, const gwas_config* cfg, void* stream, double* h_out, double* loglik_out,
                  int* evals_out) {
  if (n < 2 || q < 0 || q >= n || !phi || !y || (q && !XL) || !h_out || !(h0 > 0.0 && h0 < 1.0) || !(tol > 0.0) ||
      max_evals < 3)
    return GWAS_ERR_ARG;
  const double lo_lim = 1e-6, hi_lim = 1.0 - 1e-6;
  int evals = 0;
  double out[3];
  auto grad = [&](double h, double* g) -> int {
    int rc = reml_eval_impl(phi, n, q, XL, y, h, cfg, stream, out);
    ++evals;
    *g = out[1];
    return rc;
  };
  // bracket a sign change of dl/dh by stepping downhill-to-uphill from h0
  double a = h0, ga;
  int rc = grad(a, &ga);
  if (rc != GWAS_OK) return rc;
  double step = 0.05, b = a, gb = ga;
  while (evals < max_evals) {
    b = std::min(hi_lim, std::max(lo_lim, a + (ga > 0.0 ? step : -step)));
    if ((rc = grad(b, &gb)) != GWAS_OK) return rc;
    if ((ga > 0.0) != (gb > 0.0) || b == lo_lim || b == hi_lim) break;
    a = b;
    ga = gb;
    step *= 2.0;
  }
  double h = b, gh = gb;
  if ((ga > 0.0) == (gb > 0.0)) {
    h = b;  // the maximum sits on the boundary of (0, 1)
  } else {
    // Illinois (modified regula falsi) on the gradient
    int side = 0;
    while (std::fabs(b - a) > tol && evals < max_evals) {
      h = (a * gb - b * ga) / (gb - ga);
      if (!(h > std::min(a, b) && h < std::max(a, b))) h = 0.5 * (a + b);
      if ((rc = grad(h, &gh)) != GWAS_OK) return rc;
      if (gh == 0.0) { a = b = h; break; }
      if ((gh > 0.0) == (gb > 0.0)) {
        b = h; gb = gh;
        if (side == -1) ga *= 0.5;
        side = -1;
      } else {
        a = h; ga = gh;
        if (side == 1) gb *= 0.5;
        side = 1;
      }
      if (std::fabs(gh) == 0.0) break;
    }
    h = (std::fabs(ga) < std::fabs(gb)) ? a : b;
  }
  if ((rc = reml_eval_impl(phi, n, q, XL, y, h, cfg, stream, out)) != GWAS_OK) return rc;
  ++evals;
  *h_out = h;
  if (loglik_out) *loglik_out = out[0];
  if (evals_out) *evals_out = evals;
  return GWAS_OK;
}

}  // extern "C"

// ------------------------------------------------------------ batching form
struct gwas_batch {
  int ns = 0;
  int dev = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<gwas_ctx*> ctx;
  std::vector<tc::TcState*> ts;      // the studies' own split states
  std::vector<tc::TcState*> alt_ts;  // the same studies in the other tile mode (owned; built by the autotuner)
  bool use_alt = false;              // launches run on alt_ts
  std::vector<tc::TcBatchState*> tb;  // one planned launch per step of a replay
  // device slots of step j, study i at [j * ns + i]: n_pad x bs int8 input, outputs
  std::vector<int8_t*> slot;
  // device staging of 2-bit packed host columns, [j * ns + i], allocated on
  // first use: ceil(n_i / 4) rounded up to 16 bytes per column (pk_ld)
  std::vector<uint8_t*> pk;
  std::vector<int64_t> pk_ld;
  std::vector<double*> d_b, d_se;
  std::vector<int*> d_st;
  int ksteps = 0;  // steps with slots and a launch state
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<int> planned_cols;  // [j * ns + i]
  int planned_order = -1, planned_group = -1, planned_stages = 0;
  bool planned_alt = false;
  int order_mode = 0;
  int strip_group = 0;
  int stages = 8;
  int64_t launches = 0;
  int64_t launches_per_step = 0;
  // per study: the file readers' pinned buffers, kept across gwas_batch_solve_files calls
  std::vector<std::vector<void*>> file_buf;
  std::vector<int64_t> file_buf_bytes;
  std::string detail;
};

namespace {

int bfail(gwas_batch* B, int code, const char* msg, cudaError_t e = cudaSuccess) {
  if (B) B->detail = std::string(msg) + (e != cudaSuccess ? std::string(": ") + cudaGetErrorString(e) : "");
  return code;
}

#define BCK(call, msg)                                                                                      \
  do {                                                                                                     \
    cudaError_t e_ = (call);                                                                               \
    if (e_ != cudaSuccess) return bfail(B, e_ == cudaErrorMemoryAllocation ? GWAS_ERR_NOMEM : GWAS_ERR_CUDA, msg, e_); \
  } while (0)

const std::vector<tc::TcState*>& states(const gwas_batch* B) { return B->use_alt ? B->alt_ts : B->ts; }

void drop_graph(gwas_batch* B) {
  if (B->exec) { cudaGraphExecDestroy(B->exec); B->exec = nullptr; }
  if (B->graph) { cudaGraphDestroy(B->graph); B->graph = nullptr; }
}

void drop_alt(gwas_batch* B) {
  for (auto* t : B->alt_ts) tc::destroy(t);
  B->alt_ts.clear();
}

void batch_free(gwas_batch* B) {
  if (!B) return;
  DeviceScope dscope_(B->dev);
  if (B->stream) cudaStreamSynchronize(B->stream);
  drop_graph(B);
  for (auto* p : B->slot) cudaFree(p);
  for (auto* p : B->pk) cudaFree(p);
  for (auto* p : B->d_b) cudaFree(p);
  for (auto* p : B->d_se) cudaFree(p);
  for (auto* p : B->d_st) cudaFree(p);
  for (auto& v : B->file_buf)
    for (auto* q : v) cudaFreeHost(q);
  for (auto* t : B->tb) tc::batch_destroy(t);
  drop_alt(B);
  if (B->own_stream && B->stream) cudaStreamDestroy(B->stream);
  delete B;
}

// Launch states for steps 0 .. k-1 over the current states (rebuilt when
// the tile mode changes), and the device slots of those steps.
int ensure_steps(gwas_batch* B, int k, bool rebuild) {
  if (rebuild) {
    for (auto* t : B->tb) tc::batch_destroy(t);
    B->tb.clear();
  }
  while ((int)B->tb.size() < std::max(k, B->ksteps)) {
    tc::TcBatchState* t = nullptr;
    BCK(tc::batch_create(&t, states(B).data(), B->ns), "batch state");
    BCK(tc::batch_set_stages(t, B->stages), "stages");
    B->tb.push_back(t);
  }
  for (auto* t : B->tb) BCK(tc::batch_set_stages(t, B->stages), "stages");
  for (int j = B->ksteps; j < k; ++j) {
    for (int i = 0; i < B->ns; ++i) {
      gwas_ctx* c = B->ctx[i];
      int8_t* sl = nullptr;
      double *db = nullptr, *dse = nullptr;
      int* dst = nullptr;
      BCK(dmalloc(&sl, (size_t)c->n_pad * c->bs), "slot");
      B->slot.push_back(sl);
      BCK(cudaMemsetAsync(sl, 0, (size_t)c->n_pad * c->bs, B->stream), "slot clear");
      BCK(dmalloc(&db, sizeof(double) * (size_t)c->p * c->bs), "b");
      B->d_b.push_back(db);
      BCK(dmalloc(&dse, sizeof(double) * (size_t)c->p * c->bs), "se");
      B->d_se.push_back(dse);
      BCK(dmalloc(&dst, sizeof(int) * (size_t)c->bs), "status");
      B->d_st.push_back(dst);
    }
    B->ksteps = j + 1;
  }
  return GWAS_OK;
}

// Plans every step for cols (k * ns entries) and captures the k steps -- each
// the pre-passes, one batched launch over all studies, every study's
// reductions and p x p solves -- into one CUDA graph.
int batch_capture(gwas_batch* B, const std::vector<int>& cols, int k, int order, int group) {
  const int ns = B->ns;
  const auto& ts = states(B);
  std::vector<const int8_t*> X(ns);
  std::vector<int64_t> ld(ns);
  for (int j = 0; j < k; ++j) {
    for (int i = 0; i < ns; ++i) {
      X[i] = B->slot[j * ns + i];
      ld[i] = B->ctx[i]->n_pad;
    }
    BCK(tc::batch_plan(B->tb[j], ts.data(), X.data(), ld.data(), cols.data() + j * ns, order, B->stream, group),
        "batch plan");
  }
  drop_graph(B);
  BCK(cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
  int64_t nl = 0;
  cudaError_t e = cudaSuccess;
  for (int j = 0; j < k && e == cudaSuccess; ++j) {
    e = tc::batch_launch(B->tb[j], ts.data(), B->stream, &nl);
    for (int i = 0; i < ns && e == cudaSuccess; ++i) {
      gwas_ctx* c = B->ctx[i];
      tc::TcState* t = ts[i];
      const int nc = cols[j * ns + i], o = j * ns + i;
      if (nc == 0) continue;
      if (const float* red = tc::partials(t))
        e = launch_partials_solve(red, tc::partial_groups(t), tc::partial_ld(t), c->sc, c->q, 1, nc, B->d_b[o],
                                  B->d_se[o], B->d_st[o], tc::shift_of(t), B->stream);
      else
        e = launch_reduce_solve(tc::xt_f32(t), XT_F32, tc::xt_ld(t), c->n_pad, c->W, c->n_pad, c->sc, c->q, nc,
                                B->d_b[o], B->d_se[o], B->d_st[o], B->stream, c->W32, tc::shift_of(t), c->st,
                                c->num_sms, tc::xt_reduce_map(t));
      ++nl;
    }
  }
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(B->stream, &g);
  if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return bfail(B, GWAS_ERR_CUDA, "capture", e); }
  BCK(e2, "end capture");
  B->graph = g;
  BCK(cudaGraphInstantiate(&B->exec, g, 0), "instantiate");
  B->planned_cols = cols;
  B->planned_order = order;
  B->planned_group = group;
  B->planned_stages = B->stages;
  B->planned_alt = B->use_alt;
  B->launches_per_step = nl;
  return GWAS_OK;
}

// Device staging for the packed columns of steps 0 .. k-1 (nothing half-made
// stays behind on failure: a later call retries).
int ensure_pack_staging(gwas_batch* B, int k) {
  const int need = k * B->ns;
  if ((int)B->pk.size() >= need) return GWAS_OK;
  std::vector<uint8_t*> add;
  std::vector<int64_t> add_ld;
  for (int o = (int)B->pk.size(); o < need; ++o) {
    const gwas_ctx* c = B->ctx[o % B->ns];
    const int64_t ld = (((int64_t)c->n + 3) / 4 + 15) / 16 * 16;
    uint8_t* d = nullptr;
    const cudaError_t e = dmalloc(&d, (size_t)ld * c->bs);
    if (e != cudaSuccess) {
      for (auto* q : add) cudaFree(q);
      return bfail(B, e == cudaErrorMemoryAllocation ? GWAS_ERR_NOMEM : GWAS_ERR_CUDA, "packed staging", e);
    }
    add.push_back(d);
    add_ld.push_back(ld);
  }
  B->pk.insert(B->pk.end(), add.begin(), add.end());
  B->pk_ld.insert(B->pk_ld.end(), add_ld.begin(), add_ld.end());
  return GWAS_OK;
}

// k blocks per study through one graph replay: inputs into the slots,
// the replay (recaptured when the plan changed), results out.  Pointer
// arrays are indexed [j * ns + i]; host arrays make the call synchronous.
// packed: XR holds 2-bit packed columns (ldx bytes per column, at least
// ceil(n_i / 4)), copied into the staging (host input) and unpacked into the
// int8 slots on the GPU.
int batch_step(gwas_batch* B, int k, const void* const* XR, const int64_t* ldx, const int* ncols,
               double* const* b, double* const* se, int* const* status, bool packed = false) {
  const int ns = B->ns;
  std::vector<int> cols(k * ns);
  for (int o = 0; o < k * ns; ++o) {
    gwas_ctx* c = B->ctx[o % ns];
    const int64_t width = packed ? ((int64_t)c->n + 3) / 4 : c->n;
    if (ncols[o] < 0 || ncols[o] > c->bs || (ncols[o] > 0 && (!XR[o] || !b[o] || ldx[o] < width)))
      return bfail(B, GWAS_ERR_ARG, "bad arguments to a batch solve");
    cols[o] = ncols[o];
  }
  int rc = ensure_steps(B, k, false);
  if (rc != GWAS_OK) return rc;
  if (packed && (rc = ensure_pack_staging(B, k)) != GWAS_OK) return rc;
  bool any_host = false;
  for (int o = 0; o < k * ns; ++o) {
    if (cols[o] == 0) continue;
    gwas_ctx* c = B->ctx[o % ns];
    const bool dev_in = is_device_ptr(XR[o]);
    any_host |= !dev_in;
    if (packed) {
      const uint8_t* src = static_cast<const uint8_t*>(XR[o]);
      int64_t ld = ldx[o];
      if (!dev_in) {
        BCK(cudaMemcpy2DAsync(B->pk[o], (size_t)B->pk_ld[o], src, (size_t)ldx[o], (size_t)((c->n + 3) / 4),
                              (size_t)cols[o], cudaMemcpyHostToDevice, B->stream),
            "packed input copy");
        src = B->pk[o];
        ld = B->pk_ld[o];
      }
      BCK(launch_unpack2(src, ld, c->n, cols[o], B->slot[o], c->n_pad, B->stream), "unpack");
      B->launches += 1;
    } else {
      BCK(cudaMemcpy2DAsync(B->slot[o], (size_t)c->n_pad, XR[o], (size_t)ldx[o], (size_t)c->n, (size_t)cols[o],
                            dev_in ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, B->stream),
          "input copy");
    }
  }
  if (!B->exec || cols != B->planned_cols || B->order_mode != B->planned_order ||
      B->strip_group != B->planned_group || B->stages != B->planned_stages || B->use_alt != B->planned_alt) {
    if ((rc = batch_capture(B, cols, k, B->order_mode, B->strip_group)) != GWAS_OK) return rc;
  }
  BCK(cudaGraphLaunch(B->exec, B->stream), "graph launch");
  B->launches += B->launches_per_step;
  for (int o = 0; o < k * ns; ++o) {
    if (cols[o] == 0) continue;
    gwas_ctx* c = B->ctx[o % ns];
    any_host |= !is_device_ptr(b[o]) || (se && se[o] && !is_device_ptr(se[o])) ||
                (status && status[o] && !is_device_ptr(status[o]));
    BCK(cudaMemcpyAsync(b[o], B->d_b[o], sizeof(double) * (size_t)c->p * cols[o], cudaMemcpyDefault, B->stream),
        "b out");
    if (se && se[o])
      BCK(cudaMemcpyAsync(se[o], B->d_se[o], sizeof(double) * (size_t)c->p * cols[o], cudaMemcpyDefault, B->stream),
          "se out");
    if (status && status[o])
      BCK(cudaMemcpyAsync(status[o], B->d_st[o], sizeof(int) * (size_t)cols[o], cudaMemcpyDefault, B->stream),
          "status out");
  }
  if (!any_host) return GWAS_OK;
  BCK(cudaStreamSynchronize(B->stream), "sync");
  for (int i = 0; i < ns; ++i) {
    int r = check_device_status(B->ctx[i]);
    if (r != GWAS_OK) return bfail(B, r, "device-side wait ran out");
  }
  return GWAS_OK;
}

// Seeded dosage columns for the autotuner: x ~ Binomial(2, f_j), f_j in
// [0.05, 0.5), from a counter-based hash of (seed, column, row) -- blocks with
// the value mix of real dosages (the tensor cores' power draw, and so the
// clock under the power cap, depends on the operand values).
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__global__ void tune_dosages_kernel(int8_t* __restrict__ X, int64_t ld, int n, int ncols, uint64_t seed) {
  const int col = blockIdx.y;
  if (col >= ncols) return;
  const double f = 0.05 + 0.45 * (double)(mix64(seed ^ (0x5A17ull << 40) ^ (uint64_t)col) >> 11) * 0x1p-53;
  const uint32_t thr = (uint32_t)(f * 4294967296.0);
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const uint64_t h = mix64(seed + ((uint64_t)col << 32) + (uint64_t)r);
    X[(int64_t)col * ld + r] = (int8_t)(((uint32_t)h < thr) + ((uint32_t)(h >> 32) < thr));
  }
}

}  // namespace

extern "C" {

int gwas_batch_create(gwas_batch** out, gwas_ctx* const* studies, int nstudies, void* stream) {
  if (!out || !studies || nstudies < 1 || nstudies > tc::kMaxBatchStudies) return GWAS_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < nstudies; ++i) {
    if (!studies[i] || !studies[i]->tcs) return GWAS_ERR_ARG;  // split-precision contexts only
    if (studies[i]->prec != studies[0]->prec || studies[i]->dev != studies[0]->dev) return GWAS_ERR_ARG;
    if (studies[i]->t != 1) return GWAS_ERR_UNSUPPORTED;  // one phenotype per study in a batch
  }
  gwas_batch* B = new gwas_batch;
  B->ns = nstudies;
  B->dev = studies[0]->dev;
  DeviceScope dscope_(B->dev);
  int rc = [&]() -> int {
    BCK(dscope_.status(), "set device");
    if (stream) {
      B->stream = static_cast<cudaStream_t>(stream);
    } else {
      BCK(cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking), "stream");
      B->own_stream = true;
    }
    for (int i = 0; i < nstudies; ++i) {
      B->ctx.push_back(studies[i]);
      B->ts.push_back(studies[i]->tcs);
    }
    int r = ensure_steps(B, 1, false);
    if (r != GWAS_OK) return r;
    BCK(cudaStreamSynchronize(B->stream), "sync");
    return GWAS_OK;
  }();
  if (rc != GWAS_OK) {
    tl_init_detail = B->detail;
    batch_free(B);
    return rc;
  }
  *out = B;
  return GWAS_OK;
}

int gwas_batch_set_order(gwas_batch* B, int order_mode) {
  if (!B || order_mode < 0 || order_mode > 1) return GWAS_ERR_ARG;
  B->order_mode = order_mode;
  return GWAS_OK;
}

int gwas_batch_solve(gwas_batch* B, const int8_t* const* XR, const int64_t* ldx, const int* ncols, double* const* b,
                     double* const* se, int* const* status) {
  if (!B || !XR || !ldx || !ncols || !b) return GWAS_ERR_ARG;
  DeviceScope dscope_(B->dev);
  BCK(dscope_.status(), "set device");
  return batch_step(B, 1, reinterpret_cast<const void* const*>(XR), ldx, ncols, b, se, status);
}

int gwas_batch_solve_k(gwas_batch* B, int k, const int8_t* const* XR, const int64_t* ldx, const int* ncols,
                       double* const* b, double* const* se, int* const* status) {
  if (!B || k < 1 || k > GWAS_BATCH_MAX_STEPS || !XR || !ldx || !ncols || !b) return GWAS_ERR_ARG;
  DeviceScope dscope_(B->dev);
  BCK(dscope_.status(), "set device");
  return batch_step(B, k, reinterpret_cast<const void* const*>(XR), ldx, ncols, b, se, status);
}

int gwas_batch_synchronize(gwas_batch* B) {
  if (!B) return GWAS_ERR_ARG;
  DeviceScope dscope_(B->dev);
  BCK(dscope_.status(), "set device");
  BCK(cudaStreamSynchronize(B->stream), "sync");
  for (int i = 0; i < B->ns; ++i) {
    int rc = check_device_status(B->ctx[i]);
    if (rc != GWAS_OK) return bfail(B, rc, "device-side wait ran out");
  }
  return GWAS_OK;
}

int gwas_batch_autotune(gwas_batch* B, int reps, int* cols_out, int* order_out, double* snps_per_s_out) {
  gwas_batch_tuning t;
  int rc = gwas_batch_autotune_ex(B, reps, &t);
  if (rc != GWAS_OK) return rc;
  if (cols_out) *cols_out = t.cols;
  if (order_out) *order_out = t.order;
  if (snps_per_s_out) *snps_per_s_out = t.snps_per_s;
  return GWAS_OK;
}

int gwas_batch_autotune_ex(gwas_batch* B, int reps, gwas_batch_tuning* out) {
  if (!B || !out || reps < 1) return GWAS_ERR_ARG;
  DeviceScope dscope_(B->dev);
  BCK(dscope_.status(), "set device");
  const int ns = B->ns;
  int maxc = 1 << 30;
  for (auto* c : B->ctx) maxc = std::min(maxc, c->bs);
  // the candidates' inputs: seeded dosage blocks of maxc columns per study
  // (device), outputs into device scratch -- each timed step is a full
  // gwas_batch_solve with device arrays
  std::vector<int8_t*> src(ns, nullptr);
  std::vector<double*> ob(ns, nullptr), os(ns, nullptr);
  std::vector<int*> ost(ns, nullptr);
  std::vector<int64_t> ld(ns);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto release = [&] {
    for (int i = 0; i < ns; ++i) {
      cudaFree(src[i]);
      cudaFree(ob[i]);
      cudaFree(os[i]);
      cudaFree(ost[i]);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  int rc = [&]() -> int {
    for (int i = 0; i < ns; ++i) {
      gwas_ctx* c = B->ctx[i];
      ld[i] = c->n_pad;
      BCK(dmalloc(&src[i], (size_t)c->n_pad * maxc), "tuning input");
      BCK(dmalloc(&ob[i], sizeof(double) * (size_t)c->p * maxc), "tuning output");
      BCK(dmalloc(&os[i], sizeof(double) * (size_t)c->p * maxc), "tuning output");
      BCK(dmalloc(&ost[i], sizeof(int) * (size_t)maxc), "tuning output");
      tune_dosages_kernel<<<dim3(8, maxc), 256, 0, B->stream>>>(src[i], ld[i], c->n, maxc,
                                                                0x243F6A8885A308D3ull + 977ull * i);
      BCK(cudaGetLastError(), "tuning input");
    }
    BCK(cudaEventCreate(&e0), "event");
    BCK(cudaEventCreate(&e1), "event");
    // tile modes: the studies' own, and for BF16x3 / TF32x3 the other of
    // {inverse form, pair product} (FP16 pieces exist in the inverse form only)
    const tc::TileMode own = tc::tile_mode(B->ts[0]);
    const bool can_alt = B->ctx[0]->prec != GWAS_F16X2 && !B->ctx[0]->single_piece &&
                         (own == tc::TILES_INVERSE || own == tc::TILES_PAIR_MMA);
    const tc::TileMode other = own == tc::TILES_INVERSE ? tc::TILES_PAIR_MMA : tc::TILES_INVERSE;
    double best = -1.0;
    gwas_batch_tuning bt{};
    for (int alt = 0; alt <= (can_alt ? 1 : 0); ++alt) {
      if (alt && B->alt_ts.empty()) {  // the studies' states in the other mode
        for (int i = 0; i < ns; ++i) {
          gwas_ctx* c = B->ctx[i];
          tc::TcState* t = nullptr;
          int64_t nl = 0;
          const tc::Split sp = c->prec == GWAS_BF16X3 ? tc::SPLIT_BF16 : tc::SPLIT_TF32;
          cudaError_t e = tc::create(&t, sp, c->Aop, c->n, c->n_pad, c->bs, c->num_sms, c->intercept, c->st,
                                     B->stream, &nl, 0, other);
          B->launches += nl;
          if (e != cudaSuccess) return bfail(B, GWAS_ERR_CUDA, "tile-mode candidate", e);
          B->alt_ts.push_back(t);
          const int nw = c->q + c->t;
          if (!c->separate_sums) BCK(tc::set_reductions(t, c->W32, w32_stride(nw - 1), nw), "reductions");
        }
        BCK(cudaStreamSynchronize(B->stream), "sync");
      }
      B->use_alt = alt != 0;
      const tc::TileMode mode = alt ? other : own;
      int r = ensure_steps(B, 1, true);
      if (r != GWAS_OK) return r;
      for (int cand = 512; cand <= maxc || (cand == 512 && maxc < 512); cand *= 2) {
        const int cc = std::min(cand, maxc);
        // inverse form: 8 or 6 operand stages (no ordering: units longest first);
        // substitution: row-panel interleaved, or study after study over all strips,
        // groups of 8 or of 4 strips
        const int nvar = mode == tc::TILES_INVERSE ? 2 : 4;
        for (int v = 0; v < nvar; ++v) {
          const int stages = mode == tc::TILES_INVERSE ? (v == 0 ? 8 : 6) : 8;
          const int order = mode == tc::TILES_INVERSE ? 0 : (v == 0 ? 0 : 1);
          const int group = mode == tc::TILES_INVERSE ? 0 : (v <= 1 ? 0 : (v == 2 ? 8 : 4));
          if (group && group >= (cc + 255) / 256) continue;
          B->stages = stages;
          B->order_mode = order;
          B->strip_group = group;
          if ((r = ensure_steps(B, 1, false)) != GWAS_OK) return r;
          std::vector<int> cols(ns, cc);
          std::vector<const void*> x(src.begin(), src.end());
          if ((r = batch_step(B, 1, x.data(), ld.data(), cols.data(), ob.data(), os.data(), ost.data())) != GWAS_OK)
            return r;  // warm-up (and capture)
          BCK(cudaEventRecord(e0, B->stream), "event");
          for (int q = 0; q < reps; ++q)
            if ((r = batch_step(B, 1, x.data(), ld.data(), cols.data(), ob.data(), os.data(), ost.data())) != GWAS_OK)
              return r;
          BCK(cudaEventRecord(e1, B->stream), "event");
          BCK(cudaEventSynchronize(e1), "event sync");
          float ms = 0.f;
          BCK(cudaEventElapsedTime(&ms, e0, e1), "elapsed");
          const double rate = (double)cc * ns * reps / (ms * 1e-3);
          if (rate > best) {
            best = rate;
            bt.cols = cc;
            bt.order = order;
            bt.strip_group = group;
            bt.stages = stages;
            bt.tile_mode = mode;
            bt.snps_per_s = rate;
          }
        }
        if (cand >= maxc) break;
      }
    }
    // keep the winner
    B->use_alt = bt.tile_mode != own;
    if (!B->use_alt) drop_alt(B);
    B->stages = bt.stages;
    B->order_mode = bt.order;
    B->strip_group = bt.strip_group;
    int r = ensure_steps(B, 1, true);
    if (r != GWAS_OK) return r;
    drop_graph(B);
    B->planned_cols.clear();
    *out = bt;
    for (int i = 0; i < ns; ++i) {
      r = check_device_status(B->ctx[i]);
      if (r != GWAS_OK) return bfail(B, r, "device-side wait ran out");
    }
    return GWAS_OK;
  }();
  BCK(cudaStreamSynchronize(B->stream), "sync");
  release();
  return rc;
}

}  // extern "C"

// The batch over files of int8 or 2-bit packed columns (ldx bytes per column).
static int batch_files_impl(gwas_batch* B, const char* const* paths, const int64_t* header_bytes, const int64_t* ldx,
                            const int64_t* col0, const int64_t* m, int cols, double* const* b_host,
                            double* const* se_host, int* const* status_host, bool packed) {
  if (!B || !paths || !header_bytes || !ldx || !col0 || !m || !b_host || cols < 1) return GWAS_ERR_ARG;
  const int ns = B->ns;
  for (int i = 0; i < ns; ++i) {
    const gwas_ctx* c = B->ctx[i];
    const int64_t width = packed ? ((int64_t)c->n + 3) / 4 : c->n;
    if (!paths[i] || header_bytes[i] < 0 || ldx[i] < width || col0[i] < 0 || m[i] < 0 || cols > c->bs ||
        (m[i] > 0 && !b_host[i]))
      return bfail(B, GWAS_ERR_ARG, "bad arguments to gwas_batch_solve_files");
  }
  DeviceScope dscope_(B->dev);
  BCK(dscope_.status(), "set device");
  std::vector<int64_t> nblk(ns);
  int64_t steps = 0;
  for (int i = 0; i < ns; ++i) {
    nblk[i] = (m[i] + cols - 1) / cols;
    steps = std::max(steps, nblk[i]);
  }
  auto cols_of = [&](int i, int64_t k) { return (int)std::min<int64_t>(cols, m[i] - k * cols); };
  std::vector<gwas_reader*> rd(ns, nullptr);
  auto close_all = [&]() {
    for (auto* r : rd) gwas_reader_close(r);
  };
  B->file_buf.resize(ns);
  B->file_buf_bytes.resize(ns, 0);
  for (int i = 0; i < ns; ++i) {
    if (nblk[i] == 0) continue;
    if (B->file_buf_bytes[i] < ldx[i] * cols) {  // (re)allocate study i's pinned read buffers
      for (auto* q : B->file_buf[i]) cudaFreeHost(q);
      B->file_buf[i].assign(3, nullptr);
      B->file_buf_bytes[i] = 0;
      for (auto& q : B->file_buf[i])
        if (cudaMallocHost(&q, (size_t)(ldx[i] * cols)) != cudaSuccess) {
          cudaGetLastError();
          close_all();
          return bfail(B, GWAS_ERR_NOMEM, "pinned read buffers");
        }
      B->file_buf_bytes[i] = ldx[i] * cols;
    }
    const int rc = reader_open_with(&rd[i], paths[i], header_bytes[i] + col0[i] * ldx[i], ldx[i] * cols, nblk[i],
                                    ldx[i] * cols_of(i, nblk[i] - 1), 3, B->file_buf[i].data());
    if (rc != GWAS_OK) {
      close_all();
      return bfail(B, rc, "cannot open a study's dosage file");
    }
  }
  std::vector<const void*> xr(ns, nullptr);
  std::vector<int> nc(ns, 0);
  std::vector<double*> bo(ns, nullptr), so(ns, nullptr);
  std::vector<int*> sto(ns, nullptr);
  int rc = GWAS_OK;
  for (int64_t k = 0; k < steps && rc == GWAS_OK; ++k) {
    for (int i = 0; i < ns && rc == GWAS_OK; ++i) {
      nc[i] = k < nblk[i] ? cols_of(i, k) : 0;
      xr[i] = nullptr;
      if (nc[i] == 0) continue;
      const void* hb = nullptr;
      int64_t got = 0;
      rc = gwas_reader_next(rd[i], &hb, &got, 120000);
      if (rc != GWAS_OK) {
        B->detail = std::string("reading a study's dosage file: ") + gwas_reader_error_detail(rd[i]);
        break;
      }
      const int p = B->ctx[i]->p;
      xr[i] = hb;
      bo[i] = b_host[i] + k * cols * p;
      so[i] = (se_host && se_host[i]) ? se_host[i] + k * cols * p : nullptr;
      sto[i] = (status_host && status_host[i]) ? status_host[i] + k * cols : nullptr;
    }
    if (rc != GWAS_OK) break;
    // host inputs and outputs: returns once the step's results are in host memory
    rc = batch_step(B, 1, xr.data(), ldx, nc.data(), bo.data(), so.data(), sto.data(), packed);
    for (int i = 0; i < ns; ++i)
      if (nc[i] > 0) gwas_reader_release(rd[i]);
  }
  close_all();
  return rc;
}

extern "C" {

int gwas_batch_solve_files(gwas_batch* B, const char* const* paths, const int64_t* header_bytes, const int64_t* ldx,
                           const int64_t* col0, const int64_t* m, int cols, double* const* b_host,
                           double* const* se_host, int* const* status_host) {
  return batch_files_impl(B, paths, header_bytes, ldx, col0, m, cols, b_host, se_host, status_host, false);
}

int gwas_batch_solve_files_packed(gwas_batch* B, const char* const* paths, const int64_t* header_bytes,
                                  const int64_t* ldp, const int64_t* col0, const int64_t* m, int cols,
                                  double* const* b_host, double* const* se_host, int* const* status_host) {
  return batch_files_impl(B, paths, header_bytes, ldp, col0, m, cols, b_host, se_host, status_host, true);
}

int64_t gwas_batch_kernel_launches(const gwas_batch* B) { return B ? B->launches : 0; }
const char* gwas_batch_last_error_detail(const gwas_batch* B) { return B ? B->detail.c_str() : ""; }
void gwas_batch_destroy(gwas_batch* B) { batch_free(B); }

}  // extern "C"

namespace {
__device__ int g_never_set = 0;  // a flag no code writes

// One thread waits for a flag or an mbarrier phase that never comes, bounded
// like the solve kernels' waits (here by limit_ns): the error word and the
// abort flag are raised on expiry and the kernel returns.
__global__ void check_timeout_kernel(int kind, long long limit_ns, gwas::DevStatus* st) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  if (kind == 1) {
    gwas::ptx::mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (kind == 0)
    gwas::ptx::bounded_wait([&] { return *reinterpret_cast<volatile const int*>(&g_never_set) != 0; }, st, limit_ns);
  else
    gwas::ptx::bounded_wait([&] { return gwas::ptx::mbar_try_wait(&bar, 0); }, st, limit_ns);
}
}  // namespace

extern "C" {

int gwas_check_timeout(gwas_ctx* ctx, int kind, int limit_us) {
  if (!ctx || (kind != 0 && kind != 1) || limit_us < 1 || limit_us > 1000000) return GWAS_ERR_ARG;
  DeviceScope dscope_(ctx->dev);
  CK(dscope_.status());
  check_timeout_kernel<<<1, 32, 0, ctx->stream>>>(kind, 1000LL * limit_us, ctx->st);
  CK(cudaGetLastError());
  ctx->launches += 1;
  return check_device_status(ctx);
}

int gwas_synchronize(gwas_ctx* ctx) {
  if (!ctx) return GWAS_ERR_ARG;
  DeviceScope dscope_(ctx->dev);
  CK(dscope_.status());
  CK(cudaStreamSynchronize(ctx->stream));
  return check_device_status(ctx);
}

int gwas_set_stream(gwas_ctx* ctx, void* stream) {
  if (!ctx) return GWAS_ERR_ARG;
  ctx->stream = static_cast<cudaStream_t>(stream);
  return GWAS_OK;
}

int gwas_get_info(const gwas_ctx* ctx, int* n, int* p, int* n_pad, int* precision, int* bs) {
  if (!ctx) return GWAS_ERR_ARG;
  if (n) *n = ctx->n;
  if (p) *p = ctx->p;
  if (n_pad) *n_pad = ctx->n_pad;
  if (precision) *precision = ctx->prec;
  if (bs) *bs = ctx->bs;
  return GWAS_OK;
}

int gwas_solve_shape(const gwas_ctx* ctx, int* ctas, int* cluster_size, int* tile_mode) {
  if (!ctx) return GWAS_ERR_ARG;
  DeviceScope dscope_(ctx->dev);
  if (dscope_.status() != cudaSuccess) {
    cudaGetLastError();
    return GWAS_ERR_CUDA;
  }
  int g = 0, cl = 1, mode = GWAS_TILES_SINGLE;
  if (ctx->tcs) {
    tc::launch_shape(ctx->tcs, &g, &cl);
    mode = static_cast<int>(tc::tile_mode(ctx->tcs));
  } else if (ctx->sliced) {
    g = exact_max_ctas(ctx->sliced);
    cl = 2;
    mode = GWAS_TILES_AUTO;
  } else {
    const int tiles = (ctx->n_pad / TB) * ((ctx->bs + F64_TN - 1) / F64_TN);
    g = trsm_f64_grid(ctx->num_sms);
    if (g > tiles) g = tiles;
  }
  if (ctas) *ctas = g;
  if (cluster_size) *cluster_size = cl;
  if (tile_mode) *tile_mode = mode;
  return GWAS_OK;
}

int64_t gwas_not_spd_index(const gwas_ctx* ctx) { return ctx ? ctx->not_spd_index : tl_init_not_spd; }

int gwas_copy_factor(gwas_ctx* ctx, double* L, int64_t ld) {
  if (!ctx || !L || ld < ctx->n) return GWAS_ERR_ARG;
  DeviceScope dscope_(ctx->dev);
  CK(dscope_.status());
  CK(cudaMemcpy2DAsync(L, sizeof(double) * (size_t)ld, ctx->L, sizeof(double) * (size_t)ctx->n_pad,
                       sizeof(double) * (size_t)ctx->n, (size_t)ctx->n, cudaMemcpyDefault, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return GWAS_OK;
}

int gwas_timing_enable(gwas_ctx* ctx, int enable) {
  if (!ctx) return GWAS_ERR_ARG;
  DeviceScope dscope_(ctx->dev);
  CK(dscope_.status());
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaStreamSynchronize(ctx->copy_stream));
  CK(cudaStreamSynchronize(ctx->out_stream));
  for (auto& mk : ctx->marks) {
    ctx->event_pool.push_back(mk.a);
    ctx->event_pool.push_back(mk.b);
  }
  ctx->marks.clear();
  ctx->timing = enable != 0;
  return GWAS_OK;
}

int gwas_timing_read(gwas_ctx* ctx, double* ms, int64_t* count) {
  if (!ctx || !ms || !count) return GWAS_ERR_ARG;
  DeviceScope dscope_(ctx->dev);
  CK(dscope_.status());
  for (int i = 0; i < GWAS_NSTAGES; ++i) { ms[i] = 0.0; count[i] = 0; }
  for (auto& mk : ctx->marks) {
    CK(cudaEventSynchronize(mk.b));
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, mk.a, mk.b));
    ms[mk.stage] += t;
    count[mk.stage] += 1;
  }
  return GWAS_OK;
}

int64_t gwas_kernel_launches(const gwas_ctx* ctx) { return ctx ? ctx->launches : 0; }

int64_t gwas_h2d_bytes(const gwas_ctx* ctx) { return ctx ? ctx->h2d_bytes : 0; }

void gwas_destroy(gwas_ctx* ctx) { free_all(ctx); }

}  // extern "C"

bool gwas::ctx_view(gwas_ctx* ctx, CtxView* v) {
  if (!ctx || !v) return false;
  v->t = ctx->t;
  v->dev = ctx->dev;
  v->num_sms = ctx->num_sms;
  v->n = ctx->n;
  v->q = ctx->q;
  v->n_pad = ctx->n_pad;
  v->P = ctx->P;
  v->stream = ctx->stream;
  v->Aop = ctx->Aop;
  v->W = ctx->W;
  v->sc = ctx->sc;
  v->st = ctx->st;
  v->launches = &ctx->launches;
  v->static_scratch = ctx->static_scratch;
  return true;
}
