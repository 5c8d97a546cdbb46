// Probe update (Eq. 4) for callers that cannot allocate device memory.
//
// Some callers own all device memory themselves and may not call
// cudaMalloc / cudaFree (or any allocating library routine): a host
// application that hands this library a fixed memory budget, a plug-in whose
// framework forbids side allocations, or code that must not take the implicit
// synchronisation an allocation can cause.  dm_probe_update_static serves them:
// it runs the same probe-update kernels as dm_run_step(DM_STEP_PROBE), but the
// reduction scratch those kernels need lives in one file-scope __device__
// array of fixed size, so the call allocates nothing.  The caller passes every
// input and output buffer.
//
// Notes for users:
//  * The array (kStaticScratchBytes = 16 MiB) is part of the library image:
//    every GPU that loads the library holds it until the process exits.
//  * Its device address is looked up on every call, with the caller's device
//    current (cudaGetSymbolAddress allocates nothing), so a device whose
//    primary context was reset in between gets the array's new address.
//  * All calls share the array.  Calls whose work overlaps on the GPU (for
//    example on two streams without ordering) race on it and give wrong
//    results; order them on one stream.
//  * The array keeps the last call's contents; everything a call needs to
//    start at zero is cleared by the call itself.
//  * The call checks the positions on the device before any kernel reads the
//    object, and reads a status word after the update, so it synchronises
//    `stream` twice and returns only once the new probe is in probe_out.  It
//    cannot be recorded into a CUDA graph: on a capturing stream it returns
//    DM_EINVAL without enqueuing anything.
//  * A bounded device wait that expired during the update (which leaves the
//    result wrong rather than hanging the GPU) is returned by that same call
//    as DM_ETIMEOUT; probe_out then holds no valid result.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>

#include "dm.h"
#include "dm_kernels.h"

namespace {

constexpr size_t kStaticScratchBytes = 16ull << 20;

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Failures are reported through dm_last_error(NULL).
int fail(int code, const std::string& msg) {
  dmk::set_global_error(msg.c_str());
  return code;
}

// Checks that every footprint lies inside the object; flags a bad one.
__global__ void k_check_positions(const int2* pos, int J, int N, int H, int W, int* bad) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < J; j += gridDim.x * blockDim.x) {
    const int2 p = pos[j];
    if (p.x < 0 || p.y < 0 || p.x > H - N || p.y > W - N) atomicOr(bad, 1);
  }
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

extern "C" int dm_probe_update_static(const float* psi, const float* object, const int32_t* positions,
                                      const float* probe_in, float* probe_out, int32_t n, int32_t modes,
                                      int32_t views, int32_t obj_h, int32_t obj_w, double denom_floor_rel,
                                      void* stream) {
  dmk::set_global_error("");
  if (!psi || !object || !positions || !probe_in || !probe_out) return fail(DM_EINVAL, "a pointer is NULL");
  if (n != 16 && n != 32 && n != 64 && n != 128 && n != 256) return fail(DM_EINVAL, "n must be 16..256, a power of 2");
  if (modes < 1 || modes > dmk::kMaxModes) return fail(DM_EINVAL, "modes must be in 1..16");
  if (views < 1 || obj_h < n || obj_w < n) return fail(DM_EINVAL, "bad views or object size");
  if (!(denom_floor_rel >= 0.0) || !std::isfinite(denom_floor_rel)) return fail(DM_EINVAL, "bad denom_floor_rel");

  const size_t nn = (size_t)n * n;
  const int probe_blocks = (int)std::min<size_t>(256, (nn + dmk::kThreads - 1) / dmk::kThreads);
  // fixed part of the layout, then as many view groups as fit
  const size_t fixed = align256(sizeof(int))                                     // status word
                       + align256(2 * (size_t)modes * nn * sizeof(double))      // numerator sums
                       + align256(nn * sizeof(double))                           // denominator sums
                       + align256(nn * sizeof(float))                            // sum_k |P_k|^2
                       + align256((size_t)probe_blocks * 2 * modes * sizeof(double))
                       + align256(sizeof(unsigned long long)) + align256(sizeof(int));
  const size_t per_group = align256((size_t)modes * nn * sizeof(float2)) + align256(nn * sizeof(double));
  if (fixed + per_group > kStaticScratchBytes)
    return fail(DM_EINVAL, "n * n * modes too large for the 16 MiB static scratch (needs " +
                               std::to_string(fixed + per_group) + " bytes)");

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s, &cap);
  if (e != cudaSuccess) return fail(DM_ECUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
  if (cap != cudaStreamCaptureStatusNone)
    return fail(DM_EINVAL, "dm_probe_update_static synchronises its stream and cannot be captured in a graph");
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(DM_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  // the host-side name of the array is not a device address: ask the runtime
  // for the array's address on the current device, on every call
  void* addr = nullptr;
  e = cudaGetSymbolAddress(&addr, g_static_scratch);
  if (e != cudaSuccess || !addr)
    return fail(DM_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  unsigned char* base = static_cast<unsigned char*>(addr);

  int num_sms = 0;
  cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (num_sms < 1) num_sms = 1;
  const int tiles = (int)((nn + dmk::probe_tile_px(modes) - 1) / dmk::probe_tile_px(modes));
  int groups = (int)((kStaticScratchBytes - fixed) / per_group);
  groups = std::max(1, std::min(groups, std::min(views, num_sms / std::gcd(tiles, num_sms))));

  size_t off = 0;
  auto carve = [&](size_t bytes) { unsigned char* p = base + off; off += align256(bytes); return p; };
  int* status = reinterpret_cast<int*>(carve(sizeof(int)));
  double* num_sum = reinterpret_cast<double*>(carve(2 * (size_t)modes * nn * sizeof(double)));
  double* den_sum = reinterpret_cast<double*>(carve(nn * sizeof(double)));
  float* p2 = reinterpret_cast<float*>(carve(nn * sizeof(float)));
  double* part = reinterpret_cast<double*>(carve((size_t)probe_blocks * 2 * modes * sizeof(double)));
  unsigned long long* dmax = reinterpret_cast<unsigned long long*>(carve(sizeof(unsigned long long)));
  int* bad = reinterpret_cast<int*>(carve(sizeof(int)));
  float2* part_num = reinterpret_cast<float2*>(carve((size_t)groups * modes * nn * sizeof(float2)));
  double* part_den = reinterpret_cast<double*>(carve((size_t)groups * nn * sizeof(double)));

  const int2* pos = reinterpret_cast<const int2*>(positions);
  // positions come from device memory: check them before any kernel reads the
  // object; the status word starts at zero for this call's bounded waits
  if ((e = cudaMemsetAsync(bad, 0, sizeof(int), s)) != cudaSuccess ||
      (e = cudaMemsetAsync(status, 0, sizeof(int), s)) != cudaSuccess)
    return fail(DM_ECUDA, cudaGetErrorString(e));
  k_check_positions<<<std::max(1, std::min(1024, (views + 255) / 256)), 256, 0, s>>>(pos, views, n, obj_h, obj_w, bad);
  int hbad = 0;
  if ((e = cudaGetLastError()) != cudaSuccess ||
      (e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return fail(DM_ECUDA, cudaGetErrorString(e));
  if (hbad) return fail(DM_EINVAL, "a footprint lies outside the object");

  dmk::ProbePartialArgs a{};
  a.N = n; a.M = modes; a.J = views; a.H = obj_h; a.W = obj_w; a.groups = groups;
  a.psi = reinterpret_cast<const float2*>(psi);
  a.obj = reinterpret_cast<const float2*>(object);
  a.pos = pos;
  a.part_num = part_num;
  a.part_den = part_den;
  a.status = status;
  if ((e = dmk::launch_probe_partial(a, num_sms, s)) != cudaSuccess) return fail(DM_ECUDA, cudaGetErrorString(e));
  if ((e = cudaMemsetAsync(dmax, 0, sizeof(unsigned long long), s)) != cudaSuccess)
    return fail(DM_ECUDA, cudaGetErrorString(e));
  dmk::ProbeFinalArgs f{};
  f.N = n; f.M = modes; f.groups = groups; f.delta_rel = (float)denom_floor_rel;
  f.part_num = part_num; f.part_den = part_den;
  f.p_start = reinterpret_cast<const float2*>(probe_in);
  f.p_new = reinterpret_cast<float2*>(probe_out);
  f.p2 = p2; f.num_sum = num_sum; f.den_sum = den_sum; f.den_max_bits = dmax; f.part = part;
  int blocks = 0;
  if ((e = dmk::launch_probe_final(f, s, &blocks)) != cudaSuccess) return fail(DM_ECUDA, cudaGetErrorString(e));
  int hstatus = 0;
  if ((e = cudaMemcpyAsync(&hstatus, status, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return fail(DM_ECUDA, cudaGetErrorString(e));
  if (hstatus & dmk::kStatusTimeout)
    return fail(DM_ETIMEOUT, "a bounded device wait of the probe update expired; probe_out is not valid");
  return DM_OK;
}
