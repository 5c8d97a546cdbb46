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
// streaming (evict-first) load and store
__device__ __forceinline__ float2 psi_ldcs(const float2* p) { return __ldcs(p); }
__device__ __forceinline__ float2 psi_ldcs(const __half2* p) { return __half22float2(__ldcs(p)); }
__device__ __forceinline__ void psi_stcs(float2* p, float2 v) { __stcs(p, v); }
__device__ __forceinline__ void psi_stcs(__half2* p, float2 v) { __stcs(p, __float22half2_rn(v)); }

}  // namespace dmk
