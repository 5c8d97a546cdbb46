// Exit-wave storage types.  The exit waves psi are complex64 (float2) in the
// FP32 form of the iteration, or complex half (__half2, round-to-nearest-
// even on every store) in the mixed-precision form, where only their storage
// is narrowed: every operation on them is FP32.  These overloads are the
// only place the two forms differ in the kernels that read or write psi.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace dmk {

__device__ __forceinline__ float2 psi_ld(const float2* p) { return *p; }
__device__ __forceinline__ float2 psi_ld(const __half2* p) { return __half22float2(*p); }
// two adjacent values (p 16-byte aligned for float2, 8-byte for __half2) in one load
__device__ __forceinline__ void psi_ld2(const float2* p, float2& a, float2& b) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  a = make_float2(v.x, v.y);
  b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void psi_ld2(const __half2* p, float2& a, float2& b) {
  const uint2 v = *reinterpret_cast<const uint2*>(p);
  a = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
  b = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
}
// streaming (evict-first) load and store
__device__ __forceinline__ float2 psi_ldcs(const float2* p) { return __ldcs(p); }
__device__ __forceinline__ float2 psi_ldcs(const __half2* p) { return __half22float2(__ldcs(p)); }
__device__ __forceinline__ void psi_stcs(float2* p, float2 v) { __stcs(p, v); }
__device__ __forceinline__ void psi_stcs(__half2* p, float2 v) { __stcs(p, __float22half2_rn(v)); }

}  // namespace dmk
