// FP32-pipe peak of the current device, measured with the library's own
// kernel: the denominator of the arithmetic roofline that bench.py reports
// beside the HBM one for the Fourier step (whose radix-16 FFTs are FP32
// adds, multiplies and fused multiply-adds).
//
// Every thread runs eight independent chains of fused multiply-adds on a
// grid of four 512-thread CTAs per SM; the rate is timed with CUDA events
// on the legacy default stream after a warm-up launch.
#include <cuda_runtime.h>

#include <string>

#include "dm.h"
#include "dm_kernels.h"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(512) k_fp32_fma(float* out, int iters, float s) {
  float x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = threadIdx.x * 1e-3f + (float)i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = fmaf(x[i], s, 0.5f);
  }
  float t = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) t += x[i];
  if (t == 1234.5f) out[0] = t;   // keeps the chains alive; never true for these inputs
}

int fail(int code, const std::string& msg) {
  dmk::set_global_error(msg.c_str());
  return code;
}

}  // namespace

extern "C" int dm_fp32_peak(double* tflops) {
  dmk::set_global_error("");
  if (!tflops) return fail(DM_EINVAL, "tflops is NULL");
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  float* out = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(float));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int grid = 4 * sms, iters = 20000;
  float ms = 0.f;
  if (e == cudaSuccess) {
    k_fp32_fma<<<grid, 512>>>(out, 200, 1.0001f);
    e = cudaDeviceSynchronize();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e0);
  if (e == cudaSuccess) {
    k_fp32_fma<<<grid, 512>>>(out, iters, 1.0001f);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  if (e != cudaSuccess) return fail(DM_ECUDA, std::string("fp32 peak: ") + cudaGetErrorString(e));
  const double flops = 2.0 * kChains * (double)iters * grid * 512;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return DM_OK;
}
