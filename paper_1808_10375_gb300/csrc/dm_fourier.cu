// Fourier step of the difference map (Eq. 3 with the constrained transform
// F_c of Sec. II), as one persistent kernel over all views and modes.
//
// For view j and mode k, with PO = P_k O(r_j + .):
//   Phi   = 2 PO - psi                         (exit-wave formation)
//   X     = DFT2(Phi)                          (unnormalised 2-D DFT)
//   X'    = X * sqrt(I_j) / (N sqrt(sum_k |X_k|^2))   (modulus projection;
//           the 1/N also turns the unnormalised pair into the orthonormal one)
//   psi'  = psi + beta (IDFT2(X') - PO)
// The 2-D transform is split into row and column passes.  Writing T = row DFT
// of Phi and T'' = inverse column DFT of X', psi' = (2 - beta) PO +
// IDFT_rows(beta T'' - T / N), so the last pass needs no second read of psi.
//
// Work items ("tasks"), all with kThreads threads:
//   R(view, row block): rows of Phi -> forward row DFT -> T in a scratch slot
//   C(view, strip group): w-column strips of all modes in shared memory ->
//       forward column DFT X, modulus, inverse column DFT of (beta s - 1/N^2) X,
//       which equals U = beta T'' - T/N since T = IDFT_cols(X) / N
//   I(view, row block): inverse row DFT of U, psi' and the object source
//       c_j = sum_k conj(P_k) psi'_k (the numerator term of Eq. 5 per view)
// A CTA takes tasks from a global counter in a software-pipelined order and
// waits (bounded) on the per-chunk completion counters of what it consumes.
// Dependencies only point to earlier tasks, which were handed to running CTAs,
// so the schedule cannot deadlock.
#include <cuda_runtime.h>

#include "dm_fft.cuh"
#include "dm_kernels.h"
#include "dm_ptx.cuh"

namespace dmk {

template <int N>
struct FCfg {
  static constexpr int R1 = FftShape<N>::R1, R2 = FftShape<N>::R2, D = R1 / R2;
  static constexpr int GROUPS = kThreads / R2;          // transforms in flight per CTA
  static constexpr int GR = GROUPS < N ? GROUPS : N;     // rows per row task
  static constexpr int XB = R1 * (R2 + 1);               // exchange buffer per transform
};

// ------------------------------------------------------------------ R task
template <int N>
__device__ __forceinline__ void row_forward(const FourierArgs& a, float2* xb, const float2* tw, int j,
                                            int jj, int rb, float2* slot) {
  using C = FCfg<N>;
  const int g = threadIdx.x / C::R2, t = threadIdx.x % C::R2;
  if (g >= C::GR) return;  // whole idle warps (GR * R2 is a multiple of 32)
  const int y = rb * C::GR + g;
  const int2 p = a.pos[j];
  const float2* orow = a.obj + (size_t)(p.x + y) * a.W + p.y;
  float2* xg = xb + g * C::XB;
  for (int k = 0; k < a.M; ++k) {
    const float2* prow = a.probe + ((size_t)k * N + y) * N;
    const float2* srow = a.psi + (((size_t)j * a.M + k) * N + y) * N;
    float2 v[C::R1];
#pragma unroll
    for (int i = 0; i < C::R1; ++i) {
      const int x = t + C::R2 * i;
      const float2 po = cmul(__ldg(prow + x), __ldg(orow + x));
      const float2 s = __ldcs(srow + x);
      v[i] = make_float2(fmaf(2.f, po.x, -s.x), fmaf(2.f, po.y, -s.y));
    }
    fft_pass1<N, false>(v, t, tw);
    __syncwarp();
#pragma unroll
    for (int k1 = 0; k1 < C::R1; ++k1) xg[k1 * (C::R2 + 1) + t] = v[p1_index<N>(k1)];
    __syncwarp();
#pragma unroll
    for (int d = 0; d < C::D; ++d)
#pragma unroll
      for (int tt = 0; tt < C::R2; ++tt) v[d * C::R2 + tt] = xg[(t + C::R2 * d) * (C::R2 + 1) + tt];
    fft_pass2<N, false>(v);
    float2* trow = slot + (((size_t)jj * a.M + k) * N + y) * N;
#pragma unroll
    for (int d = 0; d < C::D; ++d)
#pragma unroll
      for (int k2 = 0; k2 < C::R2; ++k2) __stcg(trow + t + C::R2 * d + C::R1 * k2, v[p2_index<N>(d, k2)]);
  }
}

// ------------------------------------------------------------------ I task
template <int N>
__device__ __forceinline__ void row_inverse(const FourierArgs& a, float2* xb, const float2* tw, int j,
                                            int jj, int rb, const float2* slot) {
  using C = FCfg<N>;
  const int g = threadIdx.x / C::R2, t = threadIdx.x % C::R2;
  if (g >= C::GR) return;
  const int y = rb * C::GR + g;
  const int2 p = a.pos[j];
  const float2* orow = a.obj + (size_t)(p.x + y) * a.W + p.y;
  float2* xg = xb + g * C::XB;
  // c_j accumulator for this row, after the exchange buffers; each thread
  // owns the positions its pass 2 produces, so no synchronisation is needed.
  float2* cacc = xb + C::GR * C::XB + g * N;
  const float c2b = 2.f - a.beta;
  for (int k = 0; k < a.M; ++k) {
    const float2* prow = a.probe + ((size_t)k * N + y) * N;
    float2* srow = a.psi + (((size_t)j * a.M + k) * N + y) * N;
    const float2* urow = slot + (((size_t)jj * a.M + k) * N + y) * N;
    float2 v[C::R1];
#pragma unroll
    for (int i = 0; i < C::R1; ++i) v[i] = __ldcg(urow + t + C::R2 * i);
    fft_pass1<N, true>(v, t, tw);
    __syncwarp();
#pragma unroll
    for (int k1 = 0; k1 < C::R1; ++k1) xg[k1 * (C::R2 + 1) + t] = v[p1_index<N>(k1)];
    __syncwarp();
#pragma unroll
    for (int d = 0; d < C::D; ++d)
#pragma unroll
      for (int tt = 0; tt < C::R2; ++tt) v[d * C::R2 + tt] = xg[(t + C::R2 * d) * (C::R2 + 1) + tt];
    fft_pass2<N, true>(v);
#pragma unroll
    for (int d = 0; d < C::D; ++d) {
#pragma unroll
      for (int k2 = 0; k2 < C::R2; ++k2) {
        const int x = t + C::R2 * d + C::R1 * k2;
        const float2 pk = __ldg(prow + x);
        const float2 po = cmul(pk, __ldg(orow + x));
        const float2 g2 = v[p2_index<N>(d, k2)];
        const float2 pn = make_float2(fmaf(c2b, po.x, g2.x), fmaf(c2b, po.y, g2.y));
        __stcs(srow + x, pn);
        const float2 cn = cconjmul(pk, pn);
        cacc[x] = k == 0 ? cn : cadd(cacc[x], cn);
      }
    }
  }
  float2* crow = a.cview + ((size_t)j * N + y) * N;
#pragma unroll
  for (int d = 0; d < C::D; ++d)
#pragma unroll
    for (int k2 = 0; k2 < C::R2; ++k2) {
      const int x = t + C::R2 * d + C::R1 * k2;
      __stcs(crow + x, cacc[x]);
    }
}

// Column DFTs of `ncol` padded columns in shared memory (column c starts at
// c * CS; row y sits at y + y / R2).  The exchange between the two passes
// reuses the column's own storage.
template <int N, bool INV>
__device__ __forceinline__ void column_dft(float2* colbuf, int ncol, int CS, const float2* tw) {
  using C = FCfg<N>;
  const int g = threadIdx.x / C::R2, t = threadIdx.x % C::R2;
  for (int col0 = 0; col0 < ncol; col0 += C::GROUPS) {
    const int col = col0 + g;
    const bool act = col < ncol;
    float2* base = colbuf + (size_t)(act ? col : 0) * CS;
    float2 v[C::R1];
    if (act) {
#pragma unroll
      for (int i = 0; i < C::R1; ++i) v[i] = base[t + i * (C::R2 + 1)];
      fft_pass1<N, INV>(v, t, tw);
    }
    __syncwarp();
    if (act) {
#pragma unroll
      for (int k1 = 0; k1 < C::R1; ++k1) base[k1 * (C::R2 + 1) + t] = v[p1_index<N>(k1)];
    }
    __syncwarp();
    if (act) {
#pragma unroll
      for (int d = 0; d < C::D; ++d)
#pragma unroll
        for (int tt = 0; tt < C::R2; ++tt) v[d * C::R2 + tt] = base[(t + C::R2 * d) * (C::R2 + 1) + tt];
      fft_pass2<N, INV>(v);
    }
    __syncwarp();
    if (act) {
#pragma unroll
      for (int d = 0; d < C::D; ++d)
#pragma unroll
        for (int k2 = 0; k2 < C::R2; ++k2) {
          const int yy = t + C::R2 * d + C::R1 * k2;
          base[yy + yy / C::R2] = v[p2_index<N>(d, k2)];
        }
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------------ C task
template <int N>
__device__ __forceinline__ double column_task(const FourierArgs& a, float2* colbuf, const float2* tw,
                                              int j, int jj, int sg, float2* slot) {
  using C = FCfg<N>;
  constexpr int LN = Log2<N>::v;
  const int M = a.M, lw = a.lw, w = 1 << lw, CS = a.CS;
  const int tid = threadIdx.x;
  const float invN = 1.f / (float)N;
  const float invN2 = invN * invN;
  const float beta = a.beta;
  const int tot = M << (LN + lw);
  double ef = 0.0;
  for (int si = 0; si < a.SPG; ++si) {
    const int s = sg * a.SPG + si;
    const int c0 = s << lw;
    for (int e = tid; e < tot; e += kThreads) {
      const int c = e & (w - 1), y = (e >> lw) & (N - 1), k = e >> (lw + LN);
      colbuf[(k * w + c) * CS + y + y / C::R2] =
          __ldcg(slot + ((((size_t)jj * M + k) << LN) + y) * N + c0 + c);
    }
    __syncthreads();
    column_dft<N, false>(colbuf, M * w, CS, tw);
    __syncthreads();
    // modulus projection fused with the step to U (see the header)
    const float* ist = a.istrip + (((size_t)j * a.NS + s) << (lw + LN));
    for (int pq = tid; pq < (N << lw); pq += kThreads) {
      const int c = pq >> LN, y = pq & (N - 1);
      const int off = c * CS + y + y / C::R2;
      float S = 0.f;
      for (int k = 0; k < M; ++k) S += cnorm(colbuf[k * w * CS + off]);
      const float si_ = sqrtf(__ldcs(ist + pq));
      const float ss = sqrtf(S);
      const float sc = (S > 0.f) ? (si_ / ss) * invN : 0.f;
      const float dd = fmaf(ss, invN, -si_);
      ef += (double)(dd * dd);
      const float f = fmaf(beta, sc, -invN2);
      for (int k = 0; k < M; ++k) {
        float2& z = colbuf[k * w * CS + off];
        z = cscale(z, f);
      }
    }
    __syncthreads();
    column_dft<N, true>(colbuf, M * w, CS, tw);
    __syncthreads();
    for (int e = tid; e < tot; e += kThreads) {
      const int c = e & (w - 1), y = (e >> lw) & (N - 1), k = e >> (lw + LN);
      __stcg(slot + ((((size_t)jj * M + k) << LN) + y) * N + c0 + c, colbuf[(k * w + c) * CS + y + y / C::R2]);
    }
    __syncthreads();
  }
  return ef;
}

#ifndef DM_FOURIER_MIN_BLOCKS
#define DM_FOURIER_MIN_BLOCKS 2
#endif

template <int N>
__global__ void __launch_bounds__(kThreads, 2) k_fourier(const FourierArgs a) {
  using C = FCfg<N>;
  extern __shared__ __align__(16) float2 smem[];
  float2* tw = smem;
  float2* work = smem + N;
  __shared__ int s_task;
  __shared__ int s_skip;
  __shared__ double s_red[kThreads / 32];
  for (int i = threadIdx.x; i < N; i += kThreads) tw[i] = a.tw[i];

  int* disp = a.counters;
  int* doneR = a.counters + 1;
  int* doneC = doneR + a.nchunks;
  int* doneI = doneC + a.nchunks;
  int next = 0;
  if (threadIdx.x == 0) next = atomicAdd(disp, 1);
  const size_t slot_elems = (size_t)a.B * a.M * N * N;

  for (;;) {
    if (threadIdx.x == 0) {
      s_task = next;
      if (next < a.total_tasks) next = atomicAdd(disp, 1);
    }
    __syncthreads();
    const int task = s_task;
    if (task >= a.total_tasks) break;

    // Decode (stage, kind, chunk, local index).
    int lo = 0, hi = a.nstages;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (__ldg(a.stage_off + mid) <= task) lo = mid; else hi = mid;
    }
    const int st = lo;
    int local = task - __ldg(a.stage_off + st);
    int kind = -1, c = 0;
    if (st < a.nchunks) {
      const int nv = min(a.B, a.J - st * a.B);
      if (local < nv * a.RB) { kind = 0; c = st; } else local -= nv * a.RB;
    }
    if (kind < 0) {
      const int cc = st - a.lag;
      if (cc >= 0 && cc < a.nchunks) {
        const int nv = min(a.B, a.J - cc * a.B);
        if (local < nv * a.CG) { kind = 1; c = cc; } else local -= nv * a.CG;
      }
    }
    if (kind < 0) { kind = 2; c = st - 2 * a.lag; }

    // Wait for what this task consumes.
    if (threadIdx.x == 0) {
      bool ok = true;
      if (kind == 0) {
        if (c >= a.nslot) {
          const int cp = c - a.nslot;
          ok = spin_wait_geq(doneI + cp, min(a.B, a.J - cp * a.B) * a.RB, a.status);
        }
      } else if (kind == 1) {
        ok = spin_wait_geq(doneR + c, min(a.B, a.J - c * a.B) * a.RB, a.status);
      } else {
        ok = spin_wait_geq(doneC + c, min(a.B, a.J - c * a.B) * a.CG, a.status);
      }
      s_skip = ok ? 0 : 1;
    }
    __syncthreads();

    if (!s_skip) {
      float2* slot = a.scratch + (size_t)(c % a.nslot) * slot_elems;
      if (kind == 0) {
        const int jj = local / a.RB, rb = local % a.RB;
        row_forward<N>(a, work, tw, c * a.B + jj, jj, rb, slot);
      } else if (kind == 1) {
        const int jj = local / a.CG, sg = local % a.CG;
        const int j = c * a.B + jj;
        double ef = column_task<N>(a, work, tw, j, jj, sg, slot);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ef += __shfl_xor_sync(0xffffffffu, ef, o);
        if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = ef;
        __syncthreads();
        if (threadIdx.x == 0) {
          double tot = 0.0;
          for (int i = 0; i < kThreads / 32; ++i) tot += s_red[i];
          a.ef_part[(size_t)j * a.CG + sg] = tot;
        }
      } else {
        const int jj = local / a.RB, rb = local % a.RB;
        row_inverse<N>(a, work, tw, c * a.B + jj, jj, rb, slot);
      }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd((kind == 0 ? doneR : kind == 1 ? doneC : doneI) + c, 1);
  }
}

int fourier_r2(int N) {
  switch (N) {
    case 16: return FftShape<16>::R2;
    case 32: return FftShape<32>::R2;
    case 64: return FftShape<64>::R2;
    case 128: return FftShape<128>::R2;
    case 256: return FftShape<256>::R2;
    default: return 0;
  }
}

template <int N>
static size_t smem_for(int M, int w, int CS) {
  using C = FCfg<N>;
  const size_t rows = (size_t)C::GR * (C::XB + N);
  const size_t cols = (size_t)M * w * CS;
  return sizeof(float2) * (N + (rows > cols ? rows : cols));
}

size_t fourier_smem_bytes(int N, int M, int w, int CS) {
  switch (N) {
    case 16: return smem_for<16>(M, w, CS);
    case 32: return smem_for<32>(M, w, CS);
    case 64: return smem_for<64>(M, w, CS);
    case 128: return smem_for<128>(M, w, CS);
    case 256: return smem_for<256>(M, w, CS);
    default: return 0;
  }
}

template <int N>
static const void* kernel_ptr() { return (const void*)k_fourier<N>; }

static const void* fourier_kernel(int N) {
  switch (N) {
    case 16: return kernel_ptr<16>();
    case 32: return kernel_ptr<32>();
    case 64: return kernel_ptr<64>();
    case 128: return kernel_ptr<128>();
    case 256: return kernel_ptr<256>();
    default: return nullptr;
  }
}

int fourier_occupancy(int N, size_t smem) {
  const void* f = fourier_kernel(N);
  if (!f) return 0;
  if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, kThreads, smem) != cudaSuccess) return 0;
  return nb;
}

cudaError_t launch_fourier(const FourierArgs& a, int grid, size_t smem, cudaStream_t s) {
  switch (a.N) {
    case 16: k_fourier<16><<<grid, kThreads, smem, s>>>(a); break;
    case 32: k_fourier<32><<<grid, kThreads, smem, s>>>(a); break;
    case 64: k_fourier<64><<<grid, kThreads, smem, s>>>(a); break;
    case 128: k_fourier<128><<<grid, kThreads, smem, s>>>(a); break;
    case 256: k_fourier<256><<<grid, kThreads, smem, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace dmk
