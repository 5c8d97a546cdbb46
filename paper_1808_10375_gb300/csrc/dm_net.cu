// Learned warm start: a small convolutional encoder-decoder that maps one
// recorded diffraction amplitude (128 x 128, the 4-mode workload's frame) to
// the object's amplitude and phase over the central 64 x 64 pixels of the
// view's footprint.  Its predictions, stitched over the scan, replace the
// flat starting object of the difference map (the paper notes that the
// initial guess may come from prior results, Sec. III); DM itself stays the
// judge of the result.
//
// Layers (NCHW, 3 x 3 kernels, zero padding 1), six levels, 1.96 M
// parameters:
//   encoder  1 -> 16 -> 32 -> 64 -> 128 -> 256 -> 256 channels, stride 2 each
//            (128 -> 64 -> 32 -> 16 -> 8 -> 4 -> 2 pixels), ReLU
//   decoder  nearest 2x upsampling then stride 1:
//            256 -> 256 -> 128 -> 64 -> 32 -> 16 (2 -> 4 -> ... -> 64 pixels), ReLU
//   head     16 -> 2 at 64 x 64, linear (amplitude, phase)
// Weights are BF16 in every forward and backward product (FP32 master copies
// for the Adam update); activations, gradients and accumulation are FP32.
// Training loss: the mean squared error over the two output channels, or the
// phase-gauge-invariant loss.  One view's intensities are unchanged when its
// object patch is multiplied by a constant phase factor, so the second loss
// compares each predicted complex patch z = a exp(i phi) with its target t
// after the best global phase: per sample, sum|z|^2 + sum|t|^2 - 2|S| with
// S = sum conj(z) t, averaged over the pixels of the batch.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "dm.h"
#include "dm_kernels.h"

namespace dmk {

struct NetLayer {
  int ci, co, hin, win, hout, wout, stride, up, relu;
  long long w_off, b_off;   // offsets into the flat parameter array
};


static void net_layout(std::vector<NetLayer>& L, long long& nparams) {
  const int ch[7] = {1, 16, 32, 64, 128, 256, 256};
  int h = 128;
  L.clear();
  long long off = 0;
  auto add = [&](int ci, int co, int hin, int hout, int stride, int up, int relu) {
    NetLayer l{ci, co, hin, hin, hout, hout, stride, up, relu, off, off + (long long)co * ci * 9};
    off += (long long)co * ci * 9 + co;
    L.push_back(l);
  };
  for (int i = 0; i < 6; ++i) { add(ch[i], ch[i + 1], h, h / 2, 2, 0, 1); h /= 2; }
  for (int i = 6; i > 1; --i) { add(ch[i], ch[i - 1], h, 2 * h, 1, 1, 1); h *= 2; }
  add(16, 2, 64, 64, 1, 0, 0);
  nparams = off;
}

__device__ __forceinline__ float in_at(const float* in, const NetLayer& L, int b, int ci, int Y, int X) {
  // value of the (possibly upsampled) conv input at (Y, X); zero outside
  const int hu = L.up ? 2 * L.hin : L.hin, wu = L.up ? 2 * L.win : L.win;
  if (Y < 0 || Y >= hu || X < 0 || X >= wu) return 0.f;
  const int sy = L.up ? (Y >> 1) : Y, sx = L.up ? (X >> 1) : X;
  return in[(((size_t)b * L.ci + ci) * L.hin + sy) * L.win + sx];
}

__global__ void __launch_bounds__(256) k_conv_fwd(const float* __restrict__ in, float* __restrict__ out,
                                                  const __nv_bfloat16* __restrict__ w,
                                                  const float* __restrict__ bias, NetLayer L, int B) {
  const size_t n = (size_t)B * L.co * L.hout * L.wout;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % L.wout), y = (int)((i / L.wout) % L.hout);
    const int co = (int)((i / ((size_t)L.wout * L.hout)) % L.co), b = (int)(i / ((size_t)L.wout * L.hout * L.co));
    float acc = bias[co];
    for (int ci = 0; ci < L.ci; ++ci) {
      const __nv_bfloat16* wk = w + ((size_t)co * L.ci + ci) * 9;
#pragma unroll
      for (int ky = 0; ky < 3; ++ky)
#pragma unroll
        for (int kx = 0; kx < 3; ++kx)
          acc = fmaf(__bfloat162float(wk[ky * 3 + kx]), in_at(in, L, b, ci, y * L.stride + ky - 1, x * L.stride + kx - 1),
                     acc);
    }
    out[i] = L.relu ? fmaxf(acc, 0.f) : acc;
  }
}

// gradient of the loss with respect to the layer input (low resolution when
// the layer upsamples); gout is masked by the ReLU through `out`
__global__ void __launch_bounds__(256) k_conv_bwd_data(const float* __restrict__ gout, const float* __restrict__ out,
                                                       float* __restrict__ gin, const __nv_bfloat16* __restrict__ w,
                                                       NetLayer L, int B) {
  const size_t n = (size_t)B * L.ci * L.hin * L.win;
  const int f = L.up ? 2 : 1;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int ix = (int)(i % L.win), iy = (int)((i / L.win) % L.hin);
    const int ci = (int)((i / ((size_t)L.win * L.hin)) % L.ci), b = (int)(i / ((size_t)L.win * L.hin * L.ci));
    float acc = 0.f;
    for (int sy = 0; sy < f; ++sy)
      for (int sx = 0; sx < f; ++sx) {
        const int Y = iy * f + sy, X = ix * f + sx;   // conv-input position
        for (int ky = 0; ky < 3; ++ky) {
          const int ty = Y + 1 - ky;
          if (ty < 0 || ty % L.stride) continue;
          const int y = ty / L.stride;
          if (y >= L.hout) continue;
          for (int kx = 0; kx < 3; ++kx) {
            const int tx = X + 1 - kx;
            if (tx < 0 || tx % L.stride) continue;
            const int x = tx / L.stride;
            if (x >= L.wout) continue;
            for (int co = 0; co < L.co; ++co) {
              const size_t o = (((size_t)b * L.co + co) * L.hout + y) * L.wout + x;
              float g = gout[o];
              if (L.relu && !(out[o] > 0.f)) g = 0.f;
              acc = fmaf(__bfloat162float(w[(((size_t)co * L.ci + ci) * 3 + ky) * 3 + kx]), g, acc);
            }
          }
        }
      }
    gin[i] = acc;
  }
}

// weight and bias gradients: one block per (co, ci), a fixed-order block
// reduction of the nine taps (and of the bias for ci = 0)
__global__ void __launch_bounds__(256) k_conv_bwd_w(const float* __restrict__ gout, const float* __restrict__ out,
                                                    const float* __restrict__ in, float* __restrict__ gw,
                                                    float* __restrict__ gb, NetLayer L, int B) {
  __shared__ float red[10][256 / 32];
  const int co = blockIdx.x / L.ci, ci = blockIdx.x % L.ci;
  float acc[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) acc[k] = 0.f;
  const size_t n = (size_t)B * L.hout * L.wout;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) {
    const int x = (int)(i % L.wout), y = (int)((i / L.wout) % L.hout), b = (int)(i / ((size_t)L.wout * L.hout));
    const size_t o = (((size_t)b * L.co + co) * L.hout + y) * L.wout + x;
    float g = gout[o];
    if (L.relu && !(out[o] > 0.f)) g = 0.f;
    if (g == 0.f) continue;
#pragma unroll
    for (int ky = 0; ky < 3; ++ky)
#pragma unroll
      for (int kx = 0; kx < 3; ++kx)
        acc[ky * 3 + kx] = fmaf(g, in_at(in, L, b, ci, y * L.stride + ky - 1, x * L.stride + kx - 1), acc[ky * 3 + kx]);
    acc[9] += g;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 10; ++k) {
    float v = acc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[k][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < 10) {
    float s = 0.f;
    for (int i = 0; i < (int)(blockDim.x / 32); ++i) s += red[threadIdx.x][i];
    if (threadIdx.x < 9) gw[((size_t)co * L.ci + ci) * 9 + threadIdx.x] = s;
    else if (ci == 0) gb[co] = s;
  }
}

// mean squared error: gradient 2 (y - t) / count, and the sum of squares
__global__ void __launch_bounds__(256) k_mse(const float* __restrict__ y, const float* __restrict__ t,
                                             float* __restrict__ g, size_t n, double* sum) {
  double local = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float d = y[i] - t[i];
    g[i] = 2.f * d / (float)n;
    local += (double)d * d;
  }
  for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(sum, local);
}

// Gauge-invariant loss, step 1: per sample b (one block each) the sums over
// its P pixels of conj(z) t, |z|^2 and |t|^2 in FP64, in a fixed order:
// sums[b] = {Re S, Im S, sum |z|^2, sum |t|^2}.  y and t are [B][2][P] with
// channel 0 the amplitude and channel 1 the phase.
__global__ void __launch_bounds__(256) k_gauge_sums(const float* __restrict__ y, const float* __restrict__ t,
                                                    double* __restrict__ sums, int P) {
  __shared__ double red[4][256 / 32];
  const int b = blockIdx.x;
  const float* ya = y + (size_t)b * 2 * P;
  const float* ta = t + (size_t)b * 2 * P;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    float sz, cz, st, ct;
    sincosf(ya[P + p], &sz, &cz);
    sincosf(ta[P + p], &st, &ct);
    const double za = ya[p], tb = ta[p];
    const double zr = za * cz, zi = za * sz, tr = tb * ct, ti = tb * st;
    acc[0] += zr * tr + zi * ti;   // Re conj(z) t
    acc[1] += zr * ti - zi * tr;   // Im conj(z) t
    acc[2] += za * za;
    acc[3] += tb * tb;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[k][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double v = 0.0;
    for (int i = 0; i < (int)(blockDim.x / 32); ++i) v += red[threadIdx.x][i];
    sums[(size_t)b * 4 + threadIdx.x] = v;
  }
}

// Step 2: the gradient with respect to (a, phi) of every output value, with
// w = t conj(S)/|S| (the target turned by the fitted phase) and u = exp(i phi):
// dL/da = 2 (a - Re(conj(w) u)) / (B P), dL/dphi = 2 a Im(conj(w) u) / (B P);
// where S = 0 the fitted phase is undefined and w = 0.  Thread 0 of block 0
// also adds the per-sample losses in sample order into *loss_sum.
__global__ void __launch_bounds__(256) k_gauge_grad(const float* __restrict__ y, const float* __restrict__ t,
                                                    const double* __restrict__ sums, float* __restrict__ g, int B,
                                                    int P, double* loss_sum) {
  const size_t n = (size_t)B * P;
  const float scale = 2.f / (float)n;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(i / P), p = (int)(i % P);
    const double sr = sums[(size_t)b * 4], si = sums[(size_t)b * 4 + 1];
    const double mag = sqrt(sr * sr + si * si);
    const float cr = mag > 0.0 ? (float)(sr / mag) : 0.f, ci = mag > 0.0 ? (float)(-si / mag) : 0.f;   // conj(S)/|S|
    const size_t o = (size_t)b * 2 * P + p;
    float sz, cz, st, ct;
    sincosf(y[o + P], &sz, &cz);
    sincosf(t[o + P], &st, &ct);
    const float a = y[o], tb = t[o];
    const float wr = tb * (ct * cr - st * ci), wi = tb * (ct * ci + st * cr);   // w = t c
    const float re = wr * cz + wi * sz, im = wr * sz - wi * cz;                 // conj(w) u
    g[o] = scale * (a - re);
    g[o + P] = scale * a * im;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < B; ++b) {
      const double* q = sums + (size_t)b * 4;
      s += q[2] + q[3] - 2.0 * sqrt(q[0] * q[0] + q[1] * q[1]);
    }
    *loss_sum = s;
  }
}

__global__ void __launch_bounds__(256) k_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                                              const float* __restrict__ g, __nv_bfloat16* __restrict__ pb,
                                              long long n, float lr, float c1, float c2) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi, vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
    p[i] = pi;
    pb[i] = __float2bfloat16_rn(pi);
  }
}

__global__ void __launch_bounds__(256) k_to_bf16(const float* __restrict__ p, __nv_bfloat16* __restrict__ pb,
                                                 long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    pb[i] = __float2bfloat16_rn(p[i]);
}

static int grid_of(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 152 * 16); }

}  // namespace dmk

struct dm_net {
  uint32_t magic = 0x54454E44u;   // identifies a live network ('DNET')
  std::vector<dmk::NetLayer> L;
  long long np = 0;
  int max_batch = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  float *p = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;   // FP32 master, Adam moments, gradients
  __nv_bfloat16* pb = nullptr;                                     // BF16 weights used by the kernels
  std::vector<float*> act;    // act[0] input, act[l + 1] output of layer l
  std::vector<float*> grad;   // gradient of the loss w.r.t. act[l]
  double* loss = nullptr;
  double* gauge = nullptr;    // [max_batch][4] per-sample sums of the gauge-invariant loss
  int loss_kind = DM_NET_LOSS_MSE;
  long long steps = 0;
  std::string err;
};

namespace {

int net_fail(dm_net* n, int code, const std::string& msg) {
  if (n) n->err = msg;
  dmk::set_global_error(msg.c_str());
  return code;
}

#define NET_CUDA(n, call)                                                                            \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess) return net_fail(n, DM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

size_t act_elems(const dmk::NetLayer& l, int B, bool output) {
  return output ? (size_t)B * l.co * l.hout * l.wout : (size_t)B * l.ci * l.hin * l.win;
}

int net_forward(dm_net* n, const float* x, int B) {
  NET_CUDA(n, cudaMemcpyAsync(n->act[0], x, act_elems(n->L[0], B, false) * sizeof(float), cudaMemcpyDeviceToDevice,
                              n->stream));
  for (size_t i = 0; i < n->L.size(); ++i) {
    const auto& l = n->L[i];
    dmk::k_conv_fwd<<<dmk::grid_of(act_elems(l, B, true)), 256, 0, n->stream>>>(n->act[i], n->act[i + 1], n->pb + l.w_off,
                                                                                n->p + l.b_off, l, B);
    NET_CUDA(n, cudaGetLastError());
  }
  return DM_OK;
}

// The value by which the loss sum in n->loss is divided: the mean squared
// error averages over every output value, the gauge-invariant loss over the
// pixels (two output values each).
double loss_divisor(const dm_net* n, int B) {
  const double ny = (double)act_elems(n->L.back(), B, true);
  return n->loss_kind == DM_NET_LOSS_GAUGE ? ny / 2.0 : ny;
}

// gradients of the chosen loss into n->g (and the loss sum into n->loss)
int net_backward(dm_net* n, const float* target, int B) {
  const auto& last = n->L.back();
  const size_t ny = act_elems(last, B, true);
  if (n->loss_kind == DM_NET_LOSS_GAUGE) {
    const int P = last.hout * last.wout;
    dmk::k_gauge_sums<<<B, 256, 0, n->stream>>>(n->act.back(), target, n->gauge, P);
    NET_CUDA(n, cudaGetLastError());
    dmk::k_gauge_grad<<<dmk::grid_of((size_t)B * P), 256, 0, n->stream>>>(n->act.back(), target, n->gauge,
                                                                          n->grad.back(), B, P, n->loss);
  } else {
    NET_CUDA(n, cudaMemsetAsync(n->loss, 0, sizeof(double), n->stream));
    dmk::k_mse<<<dmk::grid_of(ny), 256, 0, n->stream>>>(n->act.back(), target, n->grad.back(), ny, n->loss);
  }
  NET_CUDA(n, cudaGetLastError());
  for (int i = (int)n->L.size() - 1; i >= 0; --i) {
    const auto& l = n->L[i];
    dmk::k_conv_bwd_w<<<l.co * l.ci, 256, 0, n->stream>>>(n->grad[i + 1], n->act[i + 1], n->act[i], n->g + l.w_off,
                                                          n->g + l.b_off, l, B);
    NET_CUDA(n, cudaGetLastError());
    if (i > 0) {
      dmk::k_conv_bwd_data<<<dmk::grid_of(act_elems(l, B, false)), 256, 0, n->stream>>>(
          n->grad[i + 1], n->act[i + 1], n->grad[i], n->pb + l.w_off, l, B);
      NET_CUDA(n, cudaGetLastError());
    }
  }
  return DM_OK;
}

int check_batch(dm_net* n, int B) {
  if (!n || n->magic != 0x54454E44u) return DM_EINVAL;
  if (B < 1 || B > n->max_batch) return net_fail(n, DM_EINVAL, "batch out of range");
  NET_CUDA(n, cudaSetDevice(n->device));
  return DM_OK;
}

}  // namespace

extern "C" {

int dm_net_create(dm_net** out, int32_t max_batch, uint64_t seed) {
  if (!out) return net_fail(nullptr, DM_EINVAL, "out is NULL");
  *out = nullptr;
  if (max_batch < 1 || max_batch > 4096) return net_fail(nullptr, DM_EINVAL, "max_batch out of range");
  auto* n = new dm_net();
  dmk::net_layout(n->L, n->np);
  n->max_batch = max_batch;
  cudaGetDevice(&n->device);
  auto bail = [&](int rc) { dm_net_free(n); return rc; };
  // a blocking stream: its work is ordered after work queued on the legacy
  // default stream, where callers usually produce the inputs
  cudaError_t e = cudaStreamCreateWithFlags(&n->stream, cudaStreamDefault);
  auto alloc = [&](void** ptr, size_t bytes) {
    if (e == cudaSuccess) e = cudaMallocAsync(ptr, std::max<size_t>(bytes, 256), n->stream);
  };
  alloc((void**)&n->p, n->np * sizeof(float));
  alloc((void**)&n->m, n->np * sizeof(float));
  alloc((void**)&n->v, n->np * sizeof(float));
  alloc((void**)&n->g, n->np * sizeof(float));
  alloc((void**)&n->pb, n->np * sizeof(__nv_bfloat16));
  alloc((void**)&n->loss, sizeof(double));
  alloc((void**)&n->gauge, sizeof(double) * 4 * (size_t)max_batch);
  n->act.assign(n->L.size() + 1, nullptr);
  n->grad.assign(n->L.size() + 1, nullptr);
  for (size_t i = 0; i <= n->L.size(); ++i) {
    const size_t el = i == 0 ? act_elems(n->L[0], max_batch, false) : act_elems(n->L[i - 1], max_batch, true);
    alloc((void**)&n->act[i], el * sizeof(float));
    alloc((void**)&n->grad[i], el * sizeof(float));
  }
  if (e != cudaSuccess) return bail(net_fail(nullptr, DM_ENOMEM, std::string("network buffers: ") + cudaGetErrorString(e)));
  // He-normal weights from a counter-based generator (SplitMix64 then
  // Box-Muller), zero biases; the host fills, the device receives
  std::vector<float> h(n->np, 0.f);
  uint64_t state = seed;
  auto next = [&]() {
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return (double)((z ^ (z >> 31)) >> 11) * (1.0 / 9007199254740992.0);
  };
  for (const auto& l : n->L) {
    const double sd = sqrt(2.0 / (9.0 * l.ci));
    for (long long i = 0; i < (long long)l.co * l.ci * 9; ++i) {
      const double u1 = std::max(next(), 1e-300), u2 = next();
      h[l.w_off + i] = (float)(sd * sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2));
    }
  }
  e = cudaMemcpyAsync(n->p, h.data(), n->np * sizeof(float), cudaMemcpyHostToDevice, n->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->m, 0, n->np * sizeof(float), n->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->v, 0, n->np * sizeof(float), n->stream);
  if (e == cudaSuccess) {
    dmk::k_to_bf16<<<dmk::grid_of(n->np), 256, 0, n->stream>>>(n->p, n->pb, n->np);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
  if (e != cudaSuccess) return bail(net_fail(nullptr, DM_ECUDA, cudaGetErrorString(e)));
  *out = n;
  return DM_OK;
}

int64_t dm_net_param_count(const dm_net* n) { return n && n->magic == 0x54454E44u ? n->np : 0; }

int dm_net_get_params(dm_net* n, float* out) {
  if (!n || n->magic != 0x54454E44u || !out) return DM_EINVAL;
  NET_CUDA(n, cudaMemcpyAsync(out, n->p, n->np * sizeof(float), cudaMemcpyDeviceToHost, n->stream));
  NET_CUDA(n, cudaStreamSynchronize(n->stream));
  return DM_OK;
}

int dm_net_set_params(dm_net* n, const float* in) {
  if (!n || n->magic != 0x54454E44u || !in) return DM_EINVAL;
  NET_CUDA(n, cudaMemcpyAsync(n->p, in, n->np * sizeof(float), cudaMemcpyHostToDevice, n->stream));
  dmk::k_to_bf16<<<dmk::grid_of(n->np), 256, 0, n->stream>>>(n->p, n->pb, n->np);
  NET_CUDA(n, cudaGetLastError());
  NET_CUDA(n, cudaStreamSynchronize(n->stream));
  return DM_OK;
}

int dm_net_forward(dm_net* n, const float* x, int32_t batch, float* y) {
  int rc = check_batch(n, batch);
  if (rc) return rc;
  if (!x || !y) return net_fail(n, DM_EINVAL, "a pointer is NULL");
  if ((rc = net_forward(n, x, batch))) return rc;
  NET_CUDA(n, cudaMemcpyAsync(y, n->act.back(), act_elems(n->L.back(), batch, true) * sizeof(float),
                              cudaMemcpyDeviceToDevice, n->stream));
  NET_CUDA(n, cudaStreamSynchronize(n->stream));
  return DM_OK;
}

int dm_net_gradients(dm_net* n, const float* x, const float* target, int32_t batch, float* grads, double* loss) {
  int rc = check_batch(n, batch);
  if (rc) return rc;
  if (!x || !target || !grads) return net_fail(n, DM_EINVAL, "a pointer is NULL");
  if ((rc = net_forward(n, x, batch)) || (rc = net_backward(n, target, batch))) return rc;
  NET_CUDA(n, cudaMemcpyAsync(grads, n->g, n->np * sizeof(float), cudaMemcpyDeviceToHost, n->stream));
  double s = 0.0;
  NET_CUDA(n, cudaMemcpyAsync(&s, n->loss, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
  NET_CUDA(n, cudaStreamSynchronize(n->stream));
  if (loss) *loss = s / loss_divisor(n, batch);
  return DM_OK;
}

int dm_net_train_step(dm_net* n, const float* x, const float* target, int32_t batch, float lr, double* loss) {
  int rc = check_batch(n, batch);
  if (rc) return rc;
  if (!x || !target) return net_fail(n, DM_EINVAL, "a pointer is NULL");
  if ((rc = net_forward(n, x, batch)) || (rc = net_backward(n, target, batch))) return rc;
  n->steps++;
  const float c1 = 1.f - powf(0.9f, (float)n->steps), c2 = 1.f - powf(0.999f, (float)n->steps);
  dmk::k_adam<<<dmk::grid_of(n->np), 256, 0, n->stream>>>(n->p, n->m, n->v, n->g, n->pb, n->np, lr, c1, c2);
  NET_CUDA(n, cudaGetLastError());
  double s = 0.0;
  if (loss) NET_CUDA(n, cudaMemcpyAsync(&s, n->loss, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
  // the caller may reuse x and target once the call returns
  NET_CUDA(n, cudaStreamSynchronize(n->stream));
  if (loss) *loss = s / loss_divisor(n, batch);
  return DM_OK;
}

int dm_net_set_loss(dm_net* n, int32_t kind) {
  if (!n || n->magic != 0x54454E44u) return DM_EINVAL;
  if (kind != DM_NET_LOSS_MSE && kind != DM_NET_LOSS_GAUGE) return net_fail(n, DM_EINVAL, "unknown loss");
  n->loss_kind = kind;
  return DM_OK;
}

void dm_net_free(dm_net* n) {
  if (!n || n->magic != 0x54454E44u) return;
  n->magic = 0;
  cudaSetDevice(n->device);
  if (n->stream) {
    for (void* q : {(void*)n->p, (void*)n->m, (void*)n->v, (void*)n->g, (void*)n->pb, (void*)n->loss,
                    (void*)n->gauge})
      if (q) cudaFreeAsync(q, n->stream);
    for (float* q : n->act) if (q) cudaFreeAsync(q, n->stream);
    for (float* q : n->grad) if (q) cudaFreeAsync(q, n->stream);
    cudaStreamSynchronize(n->stream);
    cudaStreamDestroy(n->stream);
  }
  delete n;
}

}  // extern "C"
