// gwas_solve_block_static: the FP64 block solve with its scratch memory in a
// fixed device array of the library instead of memory the context allocated.
//
// Who needs it: a caller that cannot allocate device memory at the time it
// solves -- for example a host process whose device memory is fully reserved
// by another framework's caching allocator, or a service that must not call
// cudaMalloc (which can synchronize the device and fail under memory
// pressure) once it is serving.  Such a caller sets the study up once
// (gwas_init) and afterwards solves blocks with no allocation at all.
//
// The scratch is one file-scope __device__ array of GWAS_STATIC_SCRATCH_BYTES.
// Host code may not use the array's name as a device address (on the host it
// names a host-side shadow), so gwas_init, with the context's device current,
// looks the address up with cudaGetSymbolAddress (static_scratch_setup) and
// keeps it in the context; the entry point passes that pointer to the kernels.
// The lookup also loads this file's module, which is when CUDA sets the array
// aside, and the set-up loads the kernels the call launches: with CUDA's lazy
// loading both would otherwise happen at the first call, which would then
// need device memory.  The address belongs to the CUDA context that was
// current at gwas_init; a context destroyed by cudaDeviceReset takes every
// gwas context of that device with it.
#include <cuda_runtime.h>

#include <cstdint>

#include "gwas_internal.cuh"

namespace {

constexpr size_t kScratchBytes = GWAS_STATIC_SCRATCH_BYTES;
constexpr size_t kSchedBytes = 128;  // scheduler counter, then the tile flags
static_assert(sizeof(gwas::Sched) == kSchedBytes, "the tile flags follow the scheduler block");

// Per-call scratch: [scheduler counter | tile flags | padding to 256 B | X~ block (FP64)].
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

bool is_device(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

namespace gwas {

cudaError_t static_scratch_setup(void** addr) {
  *addr = nullptr;
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
  if (e != cudaSuccess) return e;
  if ((e = preload_trsm_f64_int8()) != cudaSuccess) return e;
  if ((e = preload_reduce_solve_f64()) != cudaSuccess) return e;
  *addr = p;
  return cudaSuccess;
}

}  // namespace gwas

extern "C" int gwas_solve_block_static(gwas_ctx* ctx, const int8_t* XR, int64_t ldx, int ncols, double* b,
                                       double* se, int* status) {
  using namespace gwas;
  CtxView v;
  if (!ctx_view(ctx, &v)) return GWAS_ERR_ARG;
  if (v.t != 1) return GWAS_ERR_UNSUPPORTED;  // one phenotype
  if (ncols < 0 || ldx < v.n || !XR || !b) return GWAS_ERR_ARG;
  if (ncols == 0) return GWAS_OK;
  const int C = (ncols + F64_TN - 1) / F64_TN;
  const size_t flags_bytes = sizeof(int) * (size_t)v.P * C;
  const size_t xt_off = (kSchedBytes + flags_bytes + 255) / 256 * 256;
  const size_t need = xt_off + sizeof(double) * (size_t)v.n_pad * ncols;
  if (need > kScratchBytes) return GWAS_ERR_ARG;  // beyond the fixed scratch: use gwas_solve_block
  if (!v.static_scratch) return GWAS_ERR_CUDA;

  DeviceScope scope(v.dev);
  if (scope.status() != cudaSuccess) return GWAS_ERR_CUDA;
  if (!is_device(XR) || !is_device(b) || (se && !is_device(se)) || (status && !is_device(status)))
    return GWAS_ERR_ARG;
  unsigned char* sp = static_cast<unsigned char*>(v.static_scratch);
  Sched* sched = reinterpret_cast<Sched*>(sp);
  double* Xt = reinterpret_cast<double*>(sp + xt_off);

  // the scheduler counter and tile flags must start at zero on every call
  if (cudaMemsetAsync(sp, 0, kSchedBytes + flags_bytes, v.stream) != cudaSuccess) return GWAS_ERR_CUDA;
  TrsmF64Args a{};
  a.Aop = v.Aop;
  a.lda = v.n_pad;
  a.X = XR;
  a.ldx = ldx;
  a.n = v.n;
  a.Xt = Xt;
  a.ldt = v.n_pad;
  a.P = v.P;
  a.ncols = ncols;
  a.C = C;
  a.sched = sched;
  a.st = v.st;
  if (launch_trsm_f64(a, true, v.stream, v.num_sms) != cudaSuccess) return GWAS_ERR_CUDA;
  if (launch_reduce_solve(Xt, XT_F64, v.n_pad, v.n_pad, v.W, v.n_pad, v.sc, v.q, ncols, b, se, status,
                          v.stream) != cudaSuccess)
    return GWAS_ERR_CUDA;
  *v.launches += 2;
  return GWAS_OK;
}
