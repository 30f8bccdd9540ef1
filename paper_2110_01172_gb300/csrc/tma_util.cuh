// tma_util.cuh - mbarrier and bulk tensor copy helpers (inline PTX), shared by
// the kernels that move tiles with the Tensor Memory Accelerator (the
// tensor-core DFT-GEMM and the two-pass column pass), and the host-side
// tensor-map encoder.
//
// Every wait on an mbarrier is bounded (a poll limit with a short sleep
// between polls); a wait that gives up returns false, and the caller records
// the failure in the plan's device error word instead of hanging the GPU.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

namespace gbdct {
namespace tma {

// Default bound of a wait: 2^21 polls, about half a second with the sleeps.
constexpr uint32_t kDefaultPolls = 1u << 21;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void bar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(su32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(su32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for phase `parity` of the barrier to complete, at most `polls` polls
// (try_wait: a poll may suspend the thread briefly).
__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity, uint32_t polls) {
  for (uint32_t it = 0; it < polls; ++it) {
    if (try_wait(bar, parity)) return true;
    if (it >= 16) __nanosleep(256);
  }
  return false;
}

// As bar_wait, but the first poll does not block (test_wait), so a bound of
// one poll gives up on any copy still in flight right after it was issued.
__device__ __forceinline__ bool bar_wait_from_issue(uint64_t* bar, uint32_t parity, uint32_t polls) {
  if (polls == 0) return false;
  if (test_wait(bar, parity)) return true;
  return bar_wait(bar, parity, polls - 1);
}

// Tiled tensor loads into shared memory, completing on `bar` (transaction
// bytes), with an L2 eviction-priority policy.
__device__ __forceinline__ void load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar,
                                        uint64_t pol) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(su32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(su32(bar)), "l"(pol)
      : "memory");
}
__device__ __forceinline__ void load_4d(void* dst, const CUtensorMap* map, int x, int y, int z, int w, uint64_t* bar,
                                        uint64_t pol) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%2, %3, %4, %5}], [%6], %7;" ::"r"(su32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(su32(bar)), "l"(pol)
      : "memory");
}

// Contiguous bulk copy global -> shared memory (16-byte aligned addresses,
// size a multiple of 16), completing on `bar`.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
          "r"(su32(dst)),
      "l"(src), "r"(bytes), "r"(su32(bar)), "l"(pol)
      : "memory");
}

// Tiled tensor stores from shared memory (bulk-group completion).
__device__ __forceinline__ void store_3d(const CUtensorMap* map, const void* src, int x, int y, int z, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group.L2::cache_hint"
      " [%0, {%1, %2, %3}], [%4], %5;" ::"l"(reinterpret_cast<uint64_t>(map)),
      "r"(x), "r"(y), "r"(z), "r"(su32(src)), "l"(pol)
      : "memory");
}
__device__ __forceinline__ void store_4d(const CUtensorMap* map, const void* src, int x, int y, int z, int w,
                                         uint64_t pol) {
  asm volatile(
      "cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group.L2::cache_hint"
      " [%0, {%1, %2, %3, %4}], [%5], %6;" ::"l"(reinterpret_cast<uint64_t>(map)),
      "r"(x), "r"(y), "r"(z), "r"(w), "r"(su32(src)), "l"(pol)
      : "memory");
}
__device__ __forceinline__ void commit_group() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Waits until the committed bulk stores have finished reading shared memory.
__device__ __forceinline__ void wait_group_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// Orders this thread's shared-memory writes before later bulk copies read them.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Host: the driver's cuTensorMapEncodeTiled (null if unavailable).
inline PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

}  // namespace tma
}  // namespace gbdct
