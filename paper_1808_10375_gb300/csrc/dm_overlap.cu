// Overlap projection of the difference map: the object update (Eq. 5) as a
// gather over the views that cover each object tile, staged through TMA, and
// the probe update (Eq. 4) as a two-stage deterministic reduction over views.
// Also the small kernels around them: initial exit waves (Sec. II), the
// intensity layout, sum_k |P_k|^2, and the Eq. 6 / Fourier-error reductions.
#include <algorithm>

#include <cuda.h>
#include <cuda_runtime.h>

#include "dm_fft.cuh"
#include "dm_kernels.h"
#include "dm_psi.cuh"
#include "dm_ptx.cuh"

namespace dmk {

// Fixed-order block sum of a double; every thread gets the result.
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
  return t;
}

__device__ __forceinline__ float block_max(float v, float* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  float t = 0.f;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t = fmaxf(t, sh[i]);
  return t;
}

// ---------------------------------------------------------------------------
// Object update, part 1 (Eq. 5 numerator and denominator).
// One CTA per 32x32 object tile walks the tile's list of covering views in
// ascending order.  For each view, TMA brings the 32 x 34 box of the view's
// object source c_j(u) = sum_k conj(P_k(u)) psi_j^k(u) around the tile into a
// 4-stage shared-memory ring; each thread accumulates 4 pixels:
//   num(r) += c_j(r - r_j),   den(r) += sum_k |P_k(r - r_j)|^2.
// Denominators are summed in FP32 over blocks of 32 views and in FP64 across
// blocks.  The object is never the target of an atomic; only the global max
// of den uses one (order-independent, so the result is deterministic).
// ---------------------------------------------------------------------------
constexpr int kObjBoxF2 = kObjBoxW * kObjTileH;  // float2 per stage

__global__ void __launch_bounds__(kThreads) k_obj_gather(const __grid_constant__ CUtensorMap tmap,
                                                         const ObjGatherArgs a) {
  __shared__ __align__(128) float2 box[kObjStages][kObjBoxF2];
  __shared__ __align__(8) uint64_t full[kObjStages];
  __shared__ float shm[kThreads / 32];
  __shared__ int s_abort;
  const int tile = blockIdx.x;
  const int ty0 = (tile / a.tiles_x) * kObjTileH, tx0 = (tile % a.tiles_x) * kObjTileW;
  const int v0 = a.tile_ptr[tile], nv = a.tile_ptr[tile + 1] - v0;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int N = a.N;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kObjStages; ++s) mbar_init(&full[s], 1);
    fence_mbar_init();
    s_abort = 0;
  }
  __syncthreads();

  auto issue = [&](int i) {
    const int j = __ldg(a.tile_views + v0 + i);
    const int2 p = __ldg(a.pos + j);
    const int x0e = (tx0 - p.y) & ~1;  // even complex column: 16-byte aligned TMA x
    const int s = i % kObjStages;
    mbar_arrive_expect_tx(&full[s], kObjBoxF2 * (uint32_t)sizeof(float2));
    tma_load_2d(&box[s][0], &tmap, 2 * x0e, j * N + (ty0 - p.x), &full[s]);
  };
  int issued = 0;
  if (threadIdx.x == 0) {
    for (; issued < nv && issued < kObjStages; ++issued) issue(issued);
  }

  float2 num[4];
  float den32[4];
  double den64[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) { num[m] = make_float2(0.f, 0.f); den32[m] = 0.f; den64[m] = 0.0; }

  int consumed = 0;
  for (int i = 0; i < nv; ++i) {
    const int s = i % kObjStages;
    if (threadIdx.x == 0 && !mbar_wait_bounded(&full[s], (uint32_t)((i / kObjStages) & 1), a.status))
      s_abort = 1;
    __syncthreads();
    if (s_abort) break;
    const int j = __ldg(a.tile_views + v0 + i);
    const int2 p = __ldg(a.pos + j);
    const int x0e = (tx0 - p.y) & ~1;
    const int ux = tx0 + tx - p.y;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int uy = ty0 + ty + 8 * m - p.x;
      if (uy >= 0 && uy < N && ux >= 0 && ux < N) {
        num[m] = cadd(num[m], box[s][(ty + 8 * m) * kObjBoxW + (ux - x0e)]);
        den32[m] += __ldg(a.p2 + uy * N + ux);
      }
    }
    if ((i & 31) == 31) {
#pragma unroll
      for (int m = 0; m < 4; ++m) { den64[m] += den32[m]; den32[m] = 0.f; }
    }
    consumed = i + 1;
    __syncthreads();
    if (threadIdx.x == 0 && issued < nv) { issue(issued); ++issued; }
  }
  if (s_abort) {
    // Let every copy still in flight land before the CTA exits (bounded).
    if (threadIdx.x == 0) {
      for (int i = consumed; i < issued; ++i)
        mbar_wait_bounded(&full[i % kObjStages], (uint32_t)((i / kObjStages) & 1), a.status);
    }
    __syncthreads();
  }
  float lmax = 0.f;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    den64[m] += den32[m];
    const int r = ty0 + ty + 8 * m, c = tx0 + tx;
    if (r < a.H && c < a.W) {
      const float d = (float)den64[m];
      a.num[(size_t)r * a.W + c] = num[m];
      a.den[(size_t)r * a.W + c] = d;
      if (a.den64) a.den64[(size_t)r * a.W + c] = den64[m];
      lmax = fmaxf(lmax, d);
    }
  }
  const float bm = block_max(lmax, shm);
  if (threadIdx.x == 0 && bm > 0.f) atomicMax(a.den_max_bits, __float_as_uint(bm));
}

// Object update, part 2: O = num / (den + delta) on covered pixels, the
// starting value elsewhere; Eq. 6 partial sums against the starting object.
__global__ void __launch_bounds__(kThreads) k_obj_final(const ObjFinalArgs a) {
  __shared__ double sh[kThreads / 32];
  const float delta = a.delta_rel * __uint_as_float(*a.den_max_bits);
  const size_t n = (size_t)a.H * a.W;
  double d2 = 0.0, n2 = 0.0;
  for (size_t i = (size_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (size_t)gridDim.x * kThreads) {
    const float den = a.den[i];
    const float2 o0 = a.o_start[i];
    float2 on = o0;
    if (den > 0.f) {
      const float2 nm = a.num[i];
      const float dd = den + delta;
      on = make_float2(nm.x / dd, nm.y / dd);
    }
    a.o_new[i] = on;
    const float2 df = csub(on, o0);
    d2 += (double)df.x * df.x + (double)df.y * df.y;
    n2 += (double)on.x * on.x + (double)on.y * on.y;
  }
  d2 = block_sum(d2, sh);
  n2 = block_sum(n2, sh);
  if (threadIdx.x == 0) {
    a.part[2 * blockIdx.x] = d2;
    a.part[2 * blockIdx.x + 1] = n2;
  }
}

// The same division from sums held in FP64 (view shards): the quotient is
// formed in FP64 and rounded to float once.
__global__ void __launch_bounds__(kThreads) k_obj_final64(const ObjFinal64Args a) {
  __shared__ double sh[kThreads / 32];
  const double delta = a.delta_rel * __longlong_as_double((long long)*a.den_max_bits);
  const size_t n = (size_t)a.H * a.W;
  double d2 = 0.0, n2 = 0.0;
  for (size_t i = (size_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (size_t)gridDim.x * kThreads) {
    const double den = a.den[i];
    const float2 o0 = a.o_start[i];
    float2 on = o0;
    if (den > 0.0) {
      const double2 nm = a.num[i];
      const double dd = den + delta;
      on = make_float2((float)(nm.x / dd), (float)(nm.y / dd));
    }
    a.o_new[i] = on;
    const float2 df = csub(on, o0);
    d2 += (double)df.x * df.x + (double)df.y * df.y;
    n2 += (double)on.x * on.x + (double)on.y * on.y;
  }
  d2 = block_sum(d2, sh);
  n2 = block_sum(n2, sh);
  if (threadIdx.x == 0) {
    a.part[2 * blockIdx.x] = d2;
    a.part[2 * blockIdx.x + 1] = n2;
  }
}

// c_j(u) = sum_k conj(P_k(u)) psi_j^k(u): the object source, recomputed from
// the exit waves when an inner overlap pass has changed the probe.
template <class PsiT>
__global__ void __launch_bounds__(kThreads) k_obj_source(float2* cview, const PsiT* psi,
                                                         const float2* probe, int N, int M, int J) {
  const size_t nn = (size_t)N * N;
  const size_t tot = (size_t)J * nn;
  for (size_t i = (size_t)blockIdx.x * kThreads + threadIdx.x; i < tot; i += (size_t)gridDim.x * kThreads) {
    const size_t j = i / nn, u = i % nn;
    float2 acc = make_float2(0.f, 0.f);
    for (int k = 0; k < M; ++k) acc = cadd(acc, cconjmul(__ldg(probe + k * nn + u), psi_ldcs(psi + (j * M + k) * nn + u)));
    cview[i] = acc;
  }
}

// ---------------------------------------------------------------------------
// Probe update, part 1 (Eq. 4 numerator and denominator partial sums).
// Work items are (pixel tile, view group); each thread owns PX adjacent
// pixels of the tile (read with one vector load per mode) and sums over the
// group's views
//   num_k(u) += conj(O(r_j + u)) psi_j^k(u),   den(u) += |O(r_j + u)|^2
// (num in FP32, den in FP32 over 32 views then FP64), then writes the item's
// partials.  Persistent CTAs (two per SM) stream the views through a
// shared-memory ring of probe_stages<PsiT>() views: one bulk asynchronous
// copy per mode brings the tile of psi_j^k (contiguous in memory), and each
// thread copies the object values of its own pixels with 8-byte asynchronous
// copies, so several views' reads are in flight while one is summed.  A
// view's time is set by how many views are in flight (the ring's depth)
// more than by its bytes, so complex-half exit waves, half the bytes per
// view, get a ring twice as deep in about the same shared memory.
// ---------------------------------------------------------------------------
template <int MAXM, int PX, class PsiT>
__global__ void __launch_bounds__(kThreads, 2) k_probe_partial(const ProbePartialArgs a) {
  extern __shared__ unsigned char smem_raw[];
  constexpr int STAGES = probe_stages<PsiT>();
  __shared__ __align__(8) uint64_t full[STAGES];
  constexpr int TP = PX * kThreads;  // pixels per tile
  constexpr int MS = TP * (int)sizeof(PsiT) / (int)sizeof(float2);   // float2 slots of one mode's tile
  const int N = a.N, M = a.M;
  const int nn = N * N;
  const int tiles = (nn + TP - 1) / TP;
  const int items = tiles * a.groups;
  float2* ring = reinterpret_cast<float2*>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
  const int stage_elems = M * MS + TP;  // M tiles of psi, then the object values
  if (threadIdx.x == 0) {
    for (int b = 0; b < STAGES; ++b) mbar_init(&full[b], 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t issued = 0, consumed = 0;  // views issued to / taken from the ring by this CTA

  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    const int tile = item % tiles, g = item / tiles;
    const int j0 = (int)(((long long)g * a.J) / a.groups);
    const int j1 = (int)(((long long)(g + 1) * a.J) / a.groups);
    const int nv = j1 - j0;
    const int u0 = tile * TP;
    const int npx = min(TP, nn - u0);               // a multiple of 256 (nn is)
    const uint32_t mode_bytes = (uint32_t)npx * sizeof(PsiT);   // a mode's tile of psi
    int uy[PX], ux[PX];
    bool ok[PX];
    float2 acc[PX][MAXM];
    float den32[PX];
    double den64[PX];
#pragma unroll
    for (int q = 0; q < PX; ++q) {
      const int u = u0 + PX * threadIdx.x + q;
      ok[q] = PX * (int)threadIdx.x + q < npx;
      uy[q] = u / N;
      ux[q] = u % N;
      den32[q] = 0.f;
      den64[q] = 0.0;
#pragma unroll
      for (int k = 0; k < MAXM; ++k) acc[q][k] = make_float2(0.f, 0.f);
    }
    // view i of the item into the next ring stage (every thread calls this)
    auto issue = [&](int i, int2 p) {
      float2* st = ring + (size_t)(issued % STAGES) * stage_elems;
      if (threadIdx.x == 0) {
        uint64_t* bar = &full[issued % STAGES];
        mbar_arrive_expect_tx(bar, mode_bytes * (uint32_t)M);
        const PsiT* src = static_cast<const PsiT*>(a.psi) + (size_t)(j0 + i) * M * nn + u0;
        for (int k = 0; k < M; ++k) bulk_load(st + k * MS, src + (size_t)k * nn, mode_bytes, bar);
      }
#pragma unroll
      for (int q = 0; q < PX; ++q)
        if (ok[q]) cp_async8(st + M * MS + PX * threadIdx.x + q, a.obj + (size_t)(p.x + uy[q]) * a.W + p.y + ux[q]);
      ++issued;
    };
    // prologue: STAGES - 1 views in flight (one commit group each)
    for (int i = 0; i < STAGES - 1; ++i) {
      if (i < nv) issue(i, __ldg(a.pos + j0 + i));
      cp_async_commit();
    }
    int2 p_next = (STAGES - 1 < nv) ? __ldg(a.pos + j0 + STAGES - 1) : make_int2(0, 0);
    for (int v = 0; v < nv; ++v) {
      const int b = consumed % STAGES;
      if (threadIdx.x == 0) mbar_wait_bounded(&full[b], (consumed / STAGES) & 1u, a.status);
      cp_async_wait<STAGES - 2>();
      __syncthreads();
      // the stage consumed in the previous step is free for view v + S - 1
      if (v + STAGES - 1 < nv) issue(v + STAGES - 1, p_next);
      cp_async_commit();
      if (v + STAGES < nv) p_next = __ldg(a.pos + j0 + v + STAGES);
      const float2* st = ring + (size_t)b * stage_elems;
      if constexpr (PX == 2) {
        if (ok[0]) {   // the pair is whole: npx is even
          float2 o[2];
          psi_ld2(st + M * MS + 2 * threadIdx.x, o[0], o[1]);
#pragma unroll
          for (int q = 0; q < 2; ++q) den32[q] = fmaf(o[q].x, o[q].x, fmaf(o[q].y, o[q].y, den32[q]));
#pragma unroll
          for (int k = 0; k < MAXM; ++k)
            if (k < M) {
              float2 w0, w1;
              psi_ld2(reinterpret_cast<const PsiT*>(st + k * MS) + 2 * threadIdx.x, w0, w1);
              acc[0][k] = cadd(acc[0][k], cconjmul(o[0], w0));
              acc[1][k] = cadd(acc[1][k], cconjmul(o[1], w1));
            }
        }
      } else {
#pragma unroll
        for (int q = 0; q < PX; ++q) {
          if (!ok[q]) continue;
          const float2 o = st[M * MS + PX * threadIdx.x + q];
          den32[q] = fmaf(o.x, o.x, fmaf(o.y, o.y, den32[q]));
#pragma unroll
          for (int k = 0; k < MAXM; ++k)
            if (k < M)
              acc[q][k] = cadd(acc[q][k], cconjmul(o, psi_ld(reinterpret_cast<const PsiT*>(st + k * MS) +
                                                              PX * threadIdx.x + q)));
        }
      }
      ++consumed;
      if ((v & 31) == 31) {
#pragma unroll
        for (int q = 0; q < PX; ++q) { den64[q] += den32[q]; den32[q] = 0.f; }
      }
    }
#pragma unroll
    for (int q = 0; q < PX; ++q) {
      if (!ok[q]) continue;
      const int u = u0 + PX * threadIdx.x + q;
      a.part_den[(size_t)g * nn + u] = den64[q] + den32[q];
#pragma unroll
      for (int k = 0; k < MAXM; ++k)
        if (k < M) a.part_num[((size_t)g * M + k) * nn + u] = acc[q][k];
    }
    __syncthreads();  // every thread is done with the ring before the next item refills it
  }
  // copies that a timed-out wait left in flight land before the CTA exits
  if (threadIdx.x == 0)
    while (consumed < issued) {
      mbar_wait_bounded(&full[consumed % STAGES], (consumed / STAGES) & 1u, a.status);
      ++consumed;
    }
  cp_async_wait<0>();
}

// Probe update, part 2a: FP64 sums over the view groups, in group order.
__global__ void __launch_bounds__(kThreads) k_probe_sum(const ProbeFinalArgs a) {
  __shared__ float shm[kThreads / 32];
  const int nn = a.N * a.N;
  const size_t tot = (size_t)(a.M + 1) * nn;
  double lmax = 0.0;
  for (size_t i = (size_t)blockIdx.x * kThreads + threadIdx.x; i < tot; i += (size_t)gridDim.x * kThreads) {
    if (i < (size_t)a.M * nn) {
      double re = 0.0, im = 0.0;
      for (int g = 0; g < a.groups; ++g) {
        const float2 v = a.part_num[(size_t)g * a.M * nn + i];
        re += v.x;
        im += v.y;
      }
      a.num_sum[2 * i] = re;
      a.num_sum[2 * i + 1] = im;
    } else {
      const size_t u = i - (size_t)a.M * nn;
      double d = 0.0;
      for (int g = 0; g < a.groups; ++g) d += a.part_den[(size_t)g * nn + u];
      a.den_sum[u] = d;
      lmax = fmax(lmax, d);
    }
  }
  // the max is only used through delta = delta_rel * max: a float max is ample
  const float bm = block_max((float)lmax, shm);
  if (threadIdx.x == 0 && bm > 0.f) atomicMax(a.den_max_bits, (unsigned long long)__double_as_longlong((double)bm));
}

// Probe update, part 2b: division, sum_k |P_k|^2 and Eq. 6 partials per mode.
__global__ void __launch_bounds__(kThreads) k_probe_div(const ProbeFinalArgs a) {
  __shared__ double sh[kThreads / 32];
  const int nn = a.N * a.N;
  const double delta = (double)a.delta_rel * __longlong_as_double((long long)*a.den_max_bits);
  double d2[kMaxModes], n2[kMaxModes];
#pragma unroll
  for (int k = 0; k < kMaxModes; ++k) { d2[k] = 0.0; n2[k] = 0.0; }
  for (int u = blockIdx.x * kThreads + threadIdx.x; u < nn; u += gridDim.x * kThreads) {
    const double den = a.den_sum[u];
    float p2 = 0.f;
#pragma unroll
    for (int k = 0; k < kMaxModes; ++k) {
      if (k >= a.M) break;
      const size_t i = (size_t)k * nn + u;
      const float2 p0 = a.p_start[i];
      float2 pn = p0;
      if (den > 0.0) {
        const double dd = den + delta;
        pn = make_float2((float)(a.num_sum[2 * i] / dd), (float)(a.num_sum[2 * i + 1] / dd));
      }
      a.p_new[i] = pn;
      const float2 df = csub(pn, p0);
      d2[k] += (double)df.x * df.x + (double)df.y * df.y;
      n2[k] += (double)pn.x * pn.x + (double)pn.y * pn.y;
      p2 += cnorm(pn);
    }
    a.p2[u] = p2;
  }
  const int stride = 2 * a.M;
  for (int k = 0; k < a.M; ++k) {
    const double s1 = block_sum(d2[k], sh);
    const double s2 = block_sum(n2[k], sh);
    if (threadIdx.x == 0) {
      a.part[(size_t)blockIdx.x * stride + 2 * k] = s1;
      a.part[(size_t)blockIdx.x * stride + 2 * k + 1] = s2;
    }
  }
}

// ---------------------------------------------------------------------------
// Small kernels.
// ---------------------------------------------------------------------------
// psi_j^k(u) = P_k(u) O(r_j + u): the initial fields (Sec. II, first step).
template <class PsiT>
__global__ void __launch_bounds__(kThreads) k_init_psi(PsiT* psi, const float2* probe, const float2* obj,
                                                       const int2* pos, int N, int M, int J, int W) {
  // one warp per (view, mode, row); each lane forms two adjacent values and
  // writes them with one 16-byte streaming store (N is even, rows 16-byte
  // aligned); the index arithmetic is done once per row
  const long long nrows = (long long)J * M * N;
  const int lane = threadIdx.x & 31;
  const long long nwarps = (long long)gridDim.x * (kThreads / 32);
  for (long long r = (long long)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5); r < nrows; r += nwarps) {
    const int y = (int)(r % N);
    const long long jk = r / N;
    const int k = (int)(jk % M), j = (int)(jk / M);
    const int2 p = pos[j];
    const float2* prow = probe + ((size_t)k * N + y) * N;
    const float2* orow = obj + (size_t)(p.x + y) * W + p.y;
    PsiT* dst = psi + (size_t)r * N;
    for (int x = 2 * lane; x < N; x += 64) {
      const float4 pv = *reinterpret_cast<const float4*>(prow + x);
      const float2 a = cmul(make_float2(pv.x, pv.y), orow[x]);
      const float2 b = cmul(make_float2(pv.z, pv.w), orow[x + 1]);
      if constexpr (sizeof(PsiT) == sizeof(float2)) {
        __stcs(reinterpret_cast<float4*>(dst + x), make_float4(a.x, a.y, b.x, b.y));
      } else {
        psi_stcs(dst + x, a);
        psi_stcs(dst + x + 1, b);
      }
    }
  }
}

// I[j][y][x] -> strip layout [j][s][y][c] with x = s*w + c; flags negative or
// non-finite values; per-block FP64 partial sums of I.
__global__ void __launch_bounds__(kThreads) k_intensity_layout(float* istrip, const float* inten, int N, int J,
                                                               int w, double* part, int* status) {
  __shared__ double sh[kThreads / 32];
  const size_t nn = (size_t)N * N;
  const size_t tot = (size_t)J * nn;
  double acc = 0.0;
  bool bad = false;
  for (size_t i = (size_t)blockIdx.x * kThreads + threadIdx.x; i < tot; i += (size_t)gridDim.x * kThreads) {
    const size_t j = i / nn, r = i % nn;
    const int y = (int)(r / N), x = (int)(r % N);
    const float v = inten[i];
    if (!(v >= 0.f) || isinf(v)) bad = true;
    const int s = x / w, c = x % w;
    istrip[j * nn + ((size_t)s * N + y) * w + c] = v;
    acc += (double)v;
  }
  if (bad) atomicOr(status, kStatusBadInput);
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kThreads) k_p2(float* p2, const float2* probe, int N, int M) {
  const int nn = N * N;
  for (int u = blockIdx.x * kThreads + threadIdx.x; u < nn; u += gridDim.x * kThreads) {
    float s = 0.f;
    for (int k = 0; k < M; ++k) s += cnorm(probe[(size_t)k * nn + u]);
    p2[u] = s;
  }
}

__global__ void __launch_bounds__(kThreads) k_mode_power(const float2* probe, int N, double* out) {
  __shared__ double sh[kThreads / 32];
  const int nn = N * N;
  const float2* pk = probe + (size_t)blockIdx.x * nn;
  double s = 0.0;
  for (int u = threadIdx.x; u < nn; u += kThreads) s += (double)cnorm(pk[u]);
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// out = sum_i in[i * stride + offset], i < n, in a fixed order (one CTA).
__global__ void __launch_bounds__(kThreads) k_reduce_sum(const double* in, long long n, int stride, int offset,
                                                         double* out) {
  __shared__ double sh[kThreads / 32];
  double s = 0.0;
  for (long long i = threadIdx.x; i < n; i += kThreads) s += in[i * stride + offset];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) *out = s;
}

// Eq. 6 for the object and each probe mode, the Fourier error and (when the
// Fourier step tracked it, n_psi > 0) the exit-wave change into the metrics
// ring (row = [eps_obj, fourier_err, eps_probe[0..kMaxModes-1], eps_psi]; an
// untracked eps_psi is NaN).
__global__ void __launch_bounds__(kThreads) k_metrics(const double* ef_part, long long n_ef, const double* isum,
                                                      const double* obj_part, int n_obj,
                                                      const double* probe_part, int n_probe, int M,
                                                      int probe_updated, const double* psi_part, long long n_psi,
                                                      double* ring, long long* iter, int* status) {
  __shared__ double sh[kThreads / 32];
  __shared__ int s_slot;
  // the ring slot comes from the device-side iteration counter, so that a
  // captured iteration can be replayed
  if (threadIdx.x == 0) s_slot = (int)(*iter % kMetricsRing);
  __syncthreads();
  const int slot = s_slot;
  double ef = 0.0;
  for (long long i = threadIdx.x; i < n_ef; i += kThreads) ef += ef_part[i];
  ef = block_sum(ef, sh);
  double od = 0.0, on = 0.0;
  for (int i = threadIdx.x; i < n_obj; i += kThreads) { od += obj_part[2 * i]; on += obj_part[2 * i + 1]; }
  od = block_sum(od, sh);
  on = block_sum(on, sh);
  double* row = ring + (size_t)slot * kRingRow;
  {
    double pd = 0.0, pn = 0.0;
    for (long long i = threadIdx.x; i < n_psi; i += kThreads) { pd += psi_part[2 * i]; pn += psi_part[2 * i + 1]; }
    pd = block_sum(pd, sh);
    pn = block_sum(pn, sh);
    if (threadIdx.x == 0) row[kRingPsi] = n_psi <= 0 ? nan("") : (pn > 0.0 ? sqrt(pd / pn) : 0.0);
  }
  bool bad = false;
  if (threadIdx.x == 0) {
    const double is = *isum;
    row[0] = on > 0.0 ? sqrt(od / on) : 0.0;
    row[1] = is > 0.0 ? sqrt(ef / is) : 0.0;
    bad = !isfinite(row[0]) || !isfinite(row[1]);
  }
  for (int k = 0; k < M; ++k) {
    double pd = 0.0, pn = 0.0;
    if (probe_updated) {
      for (int i = threadIdx.x; i < n_probe; i += kThreads) {
        pd += probe_part[(size_t)i * 2 * M + 2 * k];
        pn += probe_part[(size_t)i * 2 * M + 2 * k + 1];
      }
    }
    pd = block_sum(pd, sh);
    pn = block_sum(pn, sh);
    if (threadIdx.x == 0) {
      row[2 + k] = pn > 0.0 ? sqrt(pd / pn) : 0.0;
      bad = bad || !isfinite(row[2 + k]);
    }
  }
  if (threadIdx.x == 0 && bad) atomicOr(status, kStatusNonFinite);
  if (threadIdx.x == 0) *iter += 1;
}

// Self-test of the bounded device waits: a counter spin-wait on a flag that
// nothing raises, and an mbarrier wait on a phase that nothing completes.
// Each must give up after the wait limit and set kStatusTimeout in its own
// status word; ok[i] records the wait's return value (0 = gave up).
__global__ void k_wait_selftest(const int* flag, int* status, int* ok) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    ok[0] = spin_wait_geq(flag, 1, status) ? 1 : 0;
    ok[1] = mbar_wait_bounded(&bar, 0u, status + 1) ? 1 : 0;   // no arrival: phase 0 never completes
  }
}

// ---------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------
cudaError_t launch_wait_selftest(const int* flag, int* status, int* ok, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(flag, status, ok);
  return cudaGetLastError();
}

// Exit waves between complex64 and complex half (round to nearest even).
__global__ void __launch_bounds__(kThreads) k_psi_to_half(__half2* dst, const float2* src, size_t n) {
  for (size_t i = (size_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (size_t)gridDim.x * kThreads)
    dst[i] = __float22half2_rn(src[i]);
}
__global__ void __launch_bounds__(kThreads) k_psi_to_float(float2* dst, const __half2* src, size_t n) {
  for (size_t i = (size_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (size_t)gridDim.x * kThreads)
    dst[i] = __half22float2(src[i]);
}

static int grid_for(size_t work, int cap) {
  size_t g = (work + kThreads - 1) / kThreads;
  if (g < 1) g = 1;
  return (int)(g < (size_t)cap ? g : (size_t)cap);
}

cudaError_t launch_obj_gather(const void* tmap, const ObjGatherArgs& a, int ntiles, cudaStream_t s) {
  k_obj_gather<<<ntiles, kThreads, 0, s>>>(*static_cast<const CUtensorMap*>(tmap), a);
  return cudaGetLastError();
}

cudaError_t launch_obj_final(const ObjFinalArgs& a, int blocks, cudaStream_t s) {
  k_obj_final<<<blocks, kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_obj_final64(const ObjFinal64Args& a, int blocks, cudaStream_t s) {
  k_obj_final64<<<blocks, kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_obj_source(float2* cview, const void* psi, int psi16, const float2* probe, int N, int M, int J,
                              cudaStream_t s) {
  if (psi16)
    k_obj_source<<<grid_for((size_t)J * N * N, 4096), kThreads, 0, s>>>(cview, static_cast<const __half2*>(psi), probe,
                                                                       N, M, J);
  else
    k_obj_source<<<grid_for((size_t)J * N * N, 4096), kThreads, 0, s>>>(cview, static_cast<const float2*>(psi), probe,
                                                                       N, M, J);
  return cudaGetLastError();
}

cudaError_t launch_psi_convert(void* dst, const void* src, size_t n, int to_half, cudaStream_t s) {
  if (to_half) k_psi_to_half<<<grid_for(n, 8192), kThreads, 0, s>>>(static_cast<__half2*>(dst), static_cast<const float2*>(src), n);
  else k_psi_to_float<<<grid_for(n, 8192), kThreads, 0, s>>>(static_cast<float2*>(dst), static_cast<const __half2*>(src), n);
  return cudaGetLastError();
}

template <class PsiT>
static size_t probe_partial_smem_t(int M) {
  const int tp = probe_tile_px(M);
  return 128 + (size_t)probe_stages<PsiT>() * ((size_t)M * tp * sizeof(PsiT) + (size_t)tp * sizeof(float2));
}

template <int MAXM, int PX, class PsiT>
static cudaError_t probe_partial_launch(const ProbePartialArgs& a, int num_sms, cudaStream_t s) {
  const size_t smem = probe_partial_smem_t<PsiT>(a.M);
  // the limit is shared by every context using this instance: allow the
  // largest mode count the instance serves
  const void* f = (const void*)k_probe_partial<MAXM, PX, PsiT>;
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)probe_partial_smem_t<PsiT>(MAXM));
  if (e != cudaSuccess) return e;
  const int tp = PX * kThreads;
  const int items = ((a.N * a.N + tp - 1) / tp) * a.groups;
  // two CTAs per SM: one CTA's per-view barrier overlaps the other's sums
  k_probe_partial<MAXM, PX, PsiT><<<std::min(items, 2 * num_sms), kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <class PsiT>
static cudaError_t probe_partial_launch_t(const ProbePartialArgs& a, int num_sms, cudaStream_t s) {
  if (a.M <= 1) return probe_partial_launch<1, kProbePxPerThread, PsiT>(a, num_sms, s);
  if (a.M <= 2) return probe_partial_launch<2, kProbePxPerThread, PsiT>(a, num_sms, s);
  if (a.M <= 4) return probe_partial_launch<4, kProbePxPerThread, PsiT>(a, num_sms, s);
  if (a.M <= 8) return probe_partial_launch<8, kProbePxPerThread, PsiT>(a, num_sms, s);
  return probe_partial_launch<16, 1, PsiT>(a, num_sms, s);
}

int probe_tile_px(int M) { return (M > 8 ? 1 : kProbePxPerThread) * kThreads; }

size_t probe_partial_smem_bytes(int M) { return probe_partial_smem_t<float2>(M); }

// Sets the dynamic shared-memory limit of the probe-partial kernel for M
// modes ahead of any launch (so that no attribute is set while a stream is
// being captured).
template <class PsiT>
static cudaError_t prepare_probe_partial_t(int M) {
  const int maxm = M <= 1 ? 1 : M <= 2 ? 2 : M <= 4 ? 4 : M <= 8 ? 8 : 16;
  const void* f = M <= 1   ? (const void*)k_probe_partial<1, kProbePxPerThread, PsiT>
                  : M <= 2 ? (const void*)k_probe_partial<2, kProbePxPerThread, PsiT>
                  : M <= 4 ? (const void*)k_probe_partial<4, kProbePxPerThread, PsiT>
                  : M <= 8 ? (const void*)k_probe_partial<8, kProbePxPerThread, PsiT>
                           : (const void*)k_probe_partial<16, 1, PsiT>;
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)probe_partial_smem_t<PsiT>(maxm));
}

// Both exit-wave forms, so that a context may switch between them later.
cudaError_t prepare_probe_partial(int M) {
  cudaError_t e = prepare_probe_partial_t<float2>(M);
  return e == cudaSuccess ? prepare_probe_partial_t<__half2>(M) : e;
}

cudaError_t launch_probe_partial(const ProbePartialArgs& a, int num_sms, cudaStream_t s) {
  return a.psi16 ? probe_partial_launch_t<__half2>(a, num_sms, s) : probe_partial_launch_t<float2>(a, num_sms, s);
}

cudaError_t launch_probe_sum(const ProbeFinalArgs& a, cudaStream_t s) {
  k_probe_sum<<<grid_for((size_t)(a.M + 1) * (size_t)a.N * a.N, 1024), kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_probe_div(const ProbeFinalArgs& a, cudaStream_t s, int* blocks_out) {
  const int b = grid_for((size_t)a.N * a.N, 256);
  k_probe_div<<<b, kThreads, 0, s>>>(a);
  *blocks_out = b;
  return cudaGetLastError();
}

// Runs 2a and 2b; *blocks_out receives the number of partial rows of 2b.
cudaError_t launch_probe_final(const ProbeFinalArgs& a, cudaStream_t s, int* blocks_out) {
  cudaError_t e = launch_probe_sum(a, s);
  if (e != cudaSuccess) return e;
  return launch_probe_div(a, s, blocks_out);
}

// Maximum of a non-negative array into *bits (as the bit pattern of the value,
// which orders like the value for non-negative floats); *bits must start at 0.
template <class T, class B>
__global__ void __launch_bounds__(kThreads) k_max_nonneg(const T* x, size_t n, B* bits) {
  __shared__ float shm[kThreads / 32];
  float m = 0.f;
  for (size_t i = (size_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (size_t)gridDim.x * kThreads)
    m = fmaxf(m, (float)x[i]);
  const float bm = block_max(m, shm);
  if (threadIdx.x == 0 && bm > 0.f) {
    if constexpr (sizeof(B) == 4) atomicMax(reinterpret_cast<unsigned*>(bits), __float_as_uint(bm));
    else atomicMax(reinterpret_cast<unsigned long long*>(bits), (unsigned long long)__double_as_longlong((double)bm));
  }
}

cudaError_t launch_max_f32(const float* x, size_t n, unsigned* bits, cudaStream_t s) {
  k_max_nonneg<float, unsigned><<<grid_for(n, 4096), kThreads, 0, s>>>(x, n, bits);
  return cudaGetLastError();
}

cudaError_t launch_max_f64(const double* x, size_t n, unsigned long long* bits, cudaStream_t s) {
  k_max_nonneg<double, unsigned long long><<<grid_for(n, 4096), kThreads, 0, s>>>(x, n, bits);
  return cudaGetLastError();
}

cudaError_t launch_init_psi(void* psi, int psi16, const float2* probe, const float2* obj, const int2* pos, int N,
                            int M, int J, int W, cudaStream_t s) {
  const long long rows = (long long)J * M * N;
  const int blocks = (int)std::min<long long>((rows + kThreads / 32 - 1) / (kThreads / 32), 8192);
  if (psi16) k_init_psi<<<blocks, kThreads, 0, s>>>(static_cast<__half2*>(psi), probe, obj, pos, N, M, J, W);
  else k_init_psi<<<blocks, kThreads, 0, s>>>(static_cast<float2*>(psi), probe, obj, pos, N, M, J, W);
  return cudaGetLastError();
}

cudaError_t launch_intensity_layout(float* istrip, const float* inten, int N, int J, int w, double* isum_part,
                                    int* status, int* blocks_out, cudaStream_t s) {
  const int b = grid_for((size_t)J * N * N, 2048);
  k_intensity_layout<<<b, kThreads, 0, s>>>(istrip, inten, N, J, w, isum_part, status);
  *blocks_out = b;
  return cudaGetLastError();
}

cudaError_t launch_p2(float* p2, const float2* probe, int N, int M, cudaStream_t s) {
  k_p2<<<grid_for((size_t)N * N, 256), kThreads, 0, s>>>(p2, probe, N, M);
  return cudaGetLastError();
}

cudaError_t launch_reduce_sum(const double* in, long long n, int stride, int offset, double* out, cudaStream_t s) {
  k_reduce_sum<<<1, kThreads, 0, s>>>(in, n, stride, offset, out);
  return cudaGetLastError();
}

cudaError_t launch_metrics(const double* ef_part, long long n_ef, const double* isum, const double* obj_part,
                           int n_obj, const double* probe_part, int n_probe, int M, int probe_updated,
                           const double* psi_part, long long n_psi, double* ring, long long* iter, int* status,
                           cudaStream_t s) {
  k_metrics<<<1, kThreads, 0, s>>>(ef_part, n_ef, isum, obj_part, n_obj, probe_part, n_probe, M, probe_updated,
                                   psi_part, n_psi, ring, iter, status);
  return cudaGetLastError();
}

cudaError_t launch_mode_power(const float2* probe, int N, int M, double* out, cudaStream_t s) {
  k_mode_power<<<M, kThreads, 0, s>>>(probe, N, out);
  return cudaGetLastError();
}

}  // namespace dmk
