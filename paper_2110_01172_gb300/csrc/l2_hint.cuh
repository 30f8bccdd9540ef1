// l2_hint.cuh - global loads and stores with an L2 eviction-priority policy.
//
// A transform streams its input and output through L2 once, while the
// intermediate array (the column spectrum, half the size of the input) is
// written by one launch and read by the next.  Marking the streamed input and
// output "evict first" and the intermediate "evict last" lets the 129 MB L2
// keep the intermediate between the launches of one transform instead of
// writing it back to DRAM and reading it again (measured without hints at
// 4096^2: the first column step wrote its whole 64 MB output to DRAM).
// The policies are created once per thread (createpolicy) and passed to
// ld/st.global.L2::cache_hint; the hint only changes replacement priority.
// ld_once additionally skips L1 allocation for data that is read only once.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gbdct {
namespace l2 {

__device__ __forceinline__ uint64_t evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ float ld(const float* a, uint64_t pol) {
  float v;
  asm volatile("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(a), "l"(pol));
  return v;
}
__device__ __forceinline__ float2 ld(const float2* a, uint64_t pol) {
  float2 v;
  asm volatile("ld.global.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(a), "l"(pol));
  return v;
}
__device__ __forceinline__ float4 ld(const float4* a, uint64_t pol) {
  float4 v;
  asm volatile("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(a), "l"(pol));
  return v;
}

// Loads of data read exactly once: not allocated in L1, so that the streamed
// data does not evict what the CTA reuses from L1 (twiddle tables).
__device__ __forceinline__ float2 ld_once(const float2* a, uint64_t pol) {
  float2 v;
  asm volatile("ld.global.L1::no_allocate.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;"
               : "=f"(v.x), "=f"(v.y)
               : "l"(a), "l"(pol));
  return v;
}
__device__ __forceinline__ float4 ld_once(const float4* a, uint64_t pol) {
  float4 v;
  asm volatile("ld.global.L1::no_allocate.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(a), "l"(pol));
  return v;
}

__device__ __forceinline__ void st(float* a, float v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(a), "f"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st(float2* a, float2 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(a), "f"(v.x), "f"(v.y), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void st(float4* a, float4 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(a), "f"(v.x), "f"(v.y),
               "f"(v.z), "f"(v.w), "l"(pol)
               : "memory");
}

}  // namespace l2
}  // namespace gbdct
