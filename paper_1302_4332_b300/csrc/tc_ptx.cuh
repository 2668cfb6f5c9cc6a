// Inline-PTX building blocks for the sm_103a tensor-core solve: mbarriers,
// TMA tile loads, and the tcgen05 (5th-generation tensor core) instructions
// with their shared-memory and instruction descriptors.  Every wait here is
// bounded: on expiry it records DEV_ERR_TIMEOUT, raises the launch's abort
// flag and returns false, so no kernel can spin forever.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "gwas_internal.cuh"

namespace gwas {
namespace ptx {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ long long globaltimer() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool aborting(const DevStatus* st) {
  return *reinterpret_cast<const volatile int*>(&st->abort) != 0;
}

__device__ __forceinline__ void raise_timeout(DevStatus* st) {
  atomicCAS(&st->err, DEV_OK, DEV_ERR_TIMEOUT);
  atomicExch(&st->abort, 1);
}

// ------------------------------------------------------------------ mbarrier
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Polls between two looks at the abort flag and the clock in a bounded wait.
// The abort flag is a global load (hundreds of cycles): read after every poll
// it would delay the waiter's reaction to the event it waits for by that much
// (measured on the pair product, whose producer waits on tile flags: 0.986 ->
// 0.969 ms a block with the flag read every 32 polls).
constexpr uint32_t WAIT_CHECK_EVERY = 32;

// Polls `done` until it holds: true; false when the launch is aborting or after
// limit_ns (the error word and the abort flag raised).  Every poll ends by
// itself (an mbarrier try_wait returns after a bounded suspension, a flag poll
// is a load), so the wait is bounded.
template <typename Done>
__device__ __forceinline__ bool bounded_wait(Done done, DevStatus* st, long long limit_ns = WAIT_LIMIT_NS) {
  if (done()) return true;
  const long long t0 = globaltimer();
  for (uint32_t i = 1;; ++i) {
    if (done()) return true;
    if (i % WAIT_CHECK_EVERY == 0) {
      if (aborting(st)) return false;
      if (globaltimer() - t0 > limit_ns) {
        raise_timeout(st);
        return false;
      }
    }
  }
}

// Waits for the phase with the given parity to complete.  False on timeout
// or when the launch is aborting.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, DevStatus* st) {
  return bounded_wait([&] { return mbar_try_wait(bar, parity); }, st);
}

// The same with cluster-scope acquire: for barriers that a peer CTA of the
// cluster arrives on with release semantics after writing this CTA's shared
// memory (st.shared::cluster).
__device__ __forceinline__ bool mbar_try_wait_cl(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

template <bool CLUSTER>
__device__ __forceinline__ bool mbar_wait_s(uint64_t* bar, uint32_t parity, DevStatus* st) {
  return bounded_wait([&] { return CLUSTER ? mbar_try_wait_cl(bar, parity) : mbar_try_wait(bar, parity); }, st);
}

// ------------------------------------------------------------------ clusters
__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// Shared::cluster address of the location `p` of this CTA's shared memory in
// CTA `rank` of the cluster (same offset).
__device__ __forceinline__ uint32_t peer_addr(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}

__device__ __forceinline__ void st_peer_u32(uint32_t cluster_addr, uint32_t v) {
  asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(cluster_addr), "r"(v) : "memory");
}

// Arrives (release, cluster scope) on an mbarrier of another CTA of the cluster.
__device__ __forceinline__ void mbar_arrive_peer(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}

// Arrives on an mbarrier of another CTA of the cluster with the default
// (CTA-scope) semantics: a count only, for arrivals that publish no data of
// their own (the bytes of a TMA load complete on the barrier by themselves).
__device__ __forceinline__ void mbar_arrive_peer_count(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}

// Cluster-wide barrier: every thread of every CTA of the cluster.
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

// ------------------------------------------------------------- global flags
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// When `who` holds: orders this CTA's earlier generic writes (made visible to
// the thread by a CTA barrier) with other CTAs' later TMA reads, then sets
// *flag = 1 with release semantics.  One predicated sequence, no branch.
__device__ __forceinline__ void publish_flag(int* flag, bool who) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %1, 0;\n\t"
      "@p fence.proxy.async.global;\n\t"
      "@p fence.acq_rel.gpu;\n\t"
      "@p st.release.gpu.global.b32 [%0], 1;\n\t}" ::"l"(flag),
      "r"(static_cast<uint32_t>(who))
      : "memory");
}

// Waits until *flag != 0 (another CTA finished a tile).  False on timeout/abort.
__device__ __forceinline__ bool wait_flag(const int* flag, DevStatus* st) {
  if (ld_acquire(flag) != 0) return true;
  return bounded_wait(
      [&] {
        __nanosleep(100);
        return ld_acquire(flag) != 0;
      },
      st);
}

// Orders this thread's generic-proxy accesses of global memory with its
// later async-proxy (TMA) accesses, and the converse.
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ----------------------------------------------------------------------- TMA
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], "
      "[%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// Pair (cta_group::2) form: the tile lands in this CTA's shared memory and
// completes bytes on `bar_cluster`, an mbarrier of this CTA or of its peer.
__device__ __forceinline__ void tma_load_2d_pair(void* dst, const CUtensorMap* map, uint32_t bar_cluster, int x,
                                                 int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], "
      "[%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar_cluster), "r"(x), "r"(y)
      : "memory");
}

// Untiled bulk copy of `bytes` (a multiple of 16) from global memory into
// this CTA's shared memory (both addresses 16-byte aligned), completing on
// `bar`'s transaction count.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Shared -> global tile store (bulk async-group completion), and its group
// bookkeeping: commit, wait until at most N groups still read shared memory,
// wait until all groups' writes are complete.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const void* src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(smem_u32(src)), "r"(x), "r"(y)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// 16 bytes global -> shared, asynchronous (both addresses 16-byte aligned);
// visible to this thread after cp_async_wait_all().
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// ------------------------------------------------------------------- tcgen05
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, both K-major; kind::f16 (BF16 inputs) or kind::tf32.
template <bool TF32>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                    uint32_t accumulate) {
  if constexpr (TF32) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
  }
}

// Arrives once on the mbarrier when all previously issued tcgen05.mma of
// this thread have completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

// ---------------------------------------------- pair (cta_group::2) forms
// One warp of each CTA of the pair allocates together; the same columns are
// allocated in both CTAs' tensor memory.
__device__ __forceinline__ void tmem_alloc_pair(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish_pair() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D (+)= A * B^T with M = 256 over the CTA pair, issued by the even CTA: A's
// rows 0..127 and B's columns 0..N/2-1 come from the issuing CTA's shared
// memory, A's rows 128..255 and B's columns N/2.. from the peer's (same
// offsets); D's rows 0..127 land in the issuing CTA's tensor memory, rows
// 128..255 in the peer's.
template <bool TF32>
__device__ __forceinline__ void mma_pair(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
  if constexpr (TF32) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
  }
}

// Arrives on the mbarrier at `bar`'s offset in every CTA of cta_mask once all
// pair MMAs issued so far by this thread have completed.
__device__ __forceinline__ void mma_commit_pair(uint64_t* bar, uint16_t cta_mask) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"(cta_mask)
      : "memory");
}

// 32 TMEM lanes x 16 consecutive 32-bit columns: thread t of the warp gets
// lane (base lane + t), columns col .. col + 15.
__device__ __forceinline__ void tmem_ld_32x32b_x16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major operand tile stored in the
// 64-byte swizzled canonical layout (rows of 64 bytes, 8-row groups 512 bytes
// apart; tile base 512-byte aligned).  Fields: start address >> 4 (bits
// 0-13), leading-dimension byte offset >> 4 (16-29, unused for this layout,
// set to 1), stride-dimension byte offset >> 4 (32-45) = 512 >> 4, descriptor
// version 1 (bits 46-47), layout type 4 = 64-byte swizzle (61-63).
__device__ __forceinline__ uint64_t sdesc_k64(uint32_t smem_addr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((smem_addr >> 4) & 0x3FFFu);
  d |= static_cast<uint64_t>(1u) << 16;
  d |= static_cast<uint64_t>(512u >> 4) << 32;
  d |= static_cast<uint64_t>(1u) << 46;
  d |= static_cast<uint64_t>(4u) << 61;
  return d;
}

// Instruction descriptor: FP32 accumulator (bits 4-5 = 1), A and B format
// (bits 7-9, 10-12: 1 = BF16, 2 = TF32), both K-major (bits 15, 16 = 0),
// N >> 3 (bits 17-22), M >> 4 (bits 24-28).
template <bool TF32>
__host__ __device__ constexpr uint32_t idesc_f32acc(int M, int N) {
  return (1u << 4) | ((TF32 ? 2u : 1u) << 7) | ((TF32 ? 2u : 1u) << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}
// The same with FP16 A and B (format 0 of kind::f16).
__host__ __device__ constexpr uint32_t idesc_f32acc_f16(int M, int N) {
  return (1u << 4) | (static_cast<uint32_t>(N >> 3) << 17) | (static_cast<uint32_t>(M >> 4) << 24);
}

// Barrier over `count` threads that also ANDs a predicate across them: every
// thread of the group gets the same outcome, so a group never splits between
// "continue" and "give up" (which would leave the rest in a later barrier).
__device__ __forceinline__ bool group_and(int id, int count, bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred pi, po;\n\tsetp.ne.u32 pi, %1, 0;\n\t"
      "bar.red.and.pred po, %2, %3, pi;\n\tselp.u32 %0, 1, 0, po;\n\t}"
      : "=r"(r)
      : "r"(static_cast<uint32_t>(v)), "r"(id), "r"(count)
      : "memory");
  return r != 0;
}

// Named barrier over `count` threads (ids 1..15; 0 is __syncthreads).
__device__ __forceinline__ void named_bar(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// (hi, lo) + (bh, bl) as a double-FP32 pair (TwoSum on the high parts): sums
// at twice FP32's precision without B300's narrow FP64 pipe.
__device__ __forceinline__ void df_add(float& hi, float& lo, float bh, float bl) {
  const float s = hi + bh;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (bh - bb);
  const float l = lo + bl + err;
  hi = s + l;
  lo = l - (hi - s);
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start while the kernel before it still runs; griddep_wait
// blocks until that kernel has completed and its memory is visible.
// griddep_launch lets the next such kernel start once every block of this one
// has issued it (or exited).  Both are no-ops for ordinary launches.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// d0 += a * b0 and d1 += a * b1 as one packed instruction (two FP32 FMAs,
// each rounded to nearest: the same results as two fmaf).
__device__ __forceinline__ void fma2(float& d0, float& d1, float a, float b0, float b1) {
  uint64_t d, av, bv;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(d0), "f"(d1));
  asm("mov.b64 %0, {%1, %1};" : "=l"(av) : "f"(a));
  asm("mov.b64 %0, {%1, %2};" : "=l"(bv) : "f"(b0), "f"(b1));
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(av), "l"(bv));
  asm("mov.b64 {%0, %1}, %2;" : "=f"(d0), "=f"(d1) : "l"(d));
}

// After a failed (timed-out or aborted) wait: 2 ms for bulk copies already in
// flight to land, so that none writes shared memory of a retired block.
__device__ __forceinline__ void settle() {
  const long long t0 = globaltimer();
  while (globaltimer() - t0 < 2000000LL) {
  }
}

}  // namespace ptx
}  // namespace gwas
