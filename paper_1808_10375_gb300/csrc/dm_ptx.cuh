// Small inline-PTX helpers: acquire loads, bounded spin-waits, mbarriers and
// TMA tile loads.  Device-only.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dm_kernels.h"

namespace dmk {

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_volatile(const int* p) {
  return *reinterpret_cast<const volatile int*>(p);
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr uint64_t kWaitLimitNs = 1000000000ull;   // bounded waits give up after 1 s

// Spin (with back-off) until *counter >= target.  Gives up, sets
// kStatusTimeout and returns false after kWaitLimitNs, or returns false at
// once when another CTA has already flagged a timeout.  Call from one thread.
__device__ __forceinline__ bool spin_wait_geq(const int* counter, int target, int* status) {
  if (ld_acquire(counter) >= target) return true;
  const uint64_t t0 = globaltimer_ns();
  unsigned ns = 32;
  for (;;) {
    if (ld_acquire(counter) >= target) return true;
    if (ld_volatile(status) & kStatusTimeout) return false;
    if (globaltimer_ns() - t0 > kWaitLimitNs) break;
    __nanosleep(ns);
    if (ns < 256) ns <<= 1;
  }
  atomicOr(status, kStatusTimeout);
  return false;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait_parity(uint64_t* bar, uint32_t parity) {
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

// Bounded wait on an mbarrier phase; on expiry (kWaitLimitNs) sets
// kStatusTimeout and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* status) {
  if (mbar_try_wait_parity(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (;;) {
    if (mbar_try_wait_parity(bar, parity)) return true;
    if (globaltimer_ns() - t0 > kWaitLimitNs) break;
  }
  atomicOr(status, kStatusTimeout);
  return false;
}

// 2-D tiled TMA load of one box into shared memory, completing on `bar`.
// The innermost coordinate x (in elements) times the element size must be a
// multiple of 16 bytes; y may be negative or out of range (zero fill).
__device__ __forceinline__ void tma_load_2d(void* dst, const void* tmap, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

}  // namespace dmk
