// Asynchronous-copy and launch-ordering primitives of sm_90+ used by the streaming kernels:
// mbarriers with bounded waits, bulk global->shared copies that complete on an mbarrier, the
// proxy fence that orders generic shared-memory reads before a later async write, and the
// programmatic-dependent-launch controls.
#pragma once
#include <cstdint>

namespace nnc {
namespace async {

constexpr long long kWaitCycles = 4000000000LL;  // about two seconds at GB300 clocks

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}

// Makes initialised mbarriers visible to the async proxy (the bulk-copy engine).
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity; false (and `code` in *err) if it ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, int* err, int code,
                                          long long limit = kWaitCycles) {
  if (mbar_try(a, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (mbar_try(a, parity)) return true;
    if (clock64() - t0 > limit) {
      if (err) atomicCAS(err, 0, code);
      return false;
    }
  }
}

// As mbar_wait, but gives up early once *abort_flag is set (by another thread of the CTA), and
// sets it when the wait runs out.
__device__ __forceinline__ bool mbar_wait_abort(uint32_t a, uint32_t parity, int* err, int code,
                                                volatile int* abort_flag,
                                                long long limit = kWaitCycles) {
  if (mbar_try(a, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (mbar_try(a, parity)) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > limit) {
      if (err) atomicCAS(err, 0, code);
      *abort_flag = 1;
      return false;
    }
  }
}

__device__ __forceinline__ void mbar_arrive(uint32_t a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}

// 2-D tiled TMA load of one box at element coordinates (x = inner, y = outer) into `dst`.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void* map, uint32_t mbar, int x,
                                            int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
      "l"((uint64_t)map), "r"(mbar), "r"(x), "r"(y)
      : "memory");
}

// Barrier among the first `threads` threads of the CTA (named barrier `id`, 1..15).
__device__ __forceinline__ void named_sync(int id, int threads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// Thread-block clusters: rank of this CTA, a full cluster barrier (release / acquire: shared
// memory written before it is visible to the other CTAs after it), and a load from the shared
// memory of CTA `rank` of the cluster at the address that `local` has in this CTA.
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}
__device__ __forceinline__ float ld_dsmem_f32(uint32_t local, uint32_t rank) {
  uint32_t remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(rank));
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(remote) : "memory");
  return v;
}

// `bytes` (a multiple of 16) from global `src` to shared `dst` (both 16-byte aligned); the
// transaction count of mbarrier `mbar` is decremented as the bytes land.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(mbar)
      : "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses before later async-proxy
// ones (a bulk copy that overwrites a stage the warp has just read).
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Programmatic dependent launch: wait until the preceding kernel in the stream has completed and
// its writes are visible; allow the next kernel in the stream to be scheduled.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

}  // namespace async
}  // namespace nnc
