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
#include <cuda.h>
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
  static constexpr int XB = R1 * R2;                     // exchange buffer per transform (= N)
};

// ------------------------------------------------------------------ R task
// The 16 lanes of a transform stage their row of psi and of P for the next
// mode with 16-byte asynchronous copies while the current mode is computed;
// the row buffers belong to the transform, so only warp-level sync is needed.
template <int N>
__device__ __forceinline__ void row_forward(const FourierArgs& a, float2* xb, float2* stage, const float2* tw,
                                            int j, int jj, int rb, float2* slot) {
  using C = FCfg<N>;
  const int g = threadIdx.x / C::R2, t = threadIdx.x % C::R2;
  if (g >= C::GR) return;  // whole idle warps (GR * R2 is a multiple of 32)
  const int y = rb * C::GR + g;
  const int2 p = a.pos[j];
  const float2* orow = a.obj + (size_t)(p.x + y) * a.W + p.y;
  float2* xg = xb + g * C::XB;
  float2* srow_s = stage + g * N;              // staged psi row
  float2* prow_s = stage + (C::GR + g) * N;    // staged probe row
  auto issue = [&](int k) {
    const float2* src = a.psi + (((size_t)j * a.M + k) * N + y) * N;
    const float2* psrc = a.probe + ((size_t)k * N + y) * N;
    for (int q = t; q < N / 2; q += C::R2) {
      cp_async16(srow_s + 2 * q, src + 2 * q);
      cp_async16(prow_s + 2 * q, psrc + 2 * q);
    }
    cp_async_commit();
  };
  issue(0);
  for (int k = 0; k < a.M; ++k) {
    cp_async_wait<0>();
    __syncwarp();
    float2 v[C::R1];
#pragma unroll
    for (int i = 0; i < C::R1; ++i) {
      const int x = t + C::R2 * i;
      const float2 po = cmul(prow_s[x], __ldg(orow + x));
      const float2 s = srow_s[x];
      v[i] = make_float2(fmaf(2.f, po.x, -s.x), fmaf(2.f, po.y, -s.y));
    }
    __syncwarp();
    if (k + 1 < a.M) issue(k + 1);
    fft_pass1<N, false>(v, t, tw);
    __syncwarp();
#pragma unroll
    for (int k1 = 0; k1 < C::R1; ++k1) xg[k1 * C::R2 + (t ^ (k1 & (C::R2 - 1)))] = v[p1_index<N>(k1)];
    __syncwarp();
#pragma unroll
    for (int d = 0; d < C::D; ++d)
#pragma unroll
      for (int tt = 0; tt < C::R2; ++tt) v[d * C::R2 + tt] = xg[(t + C::R2 * d) * C::R2 + (tt ^ t)];
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
__device__ __forceinline__ void row_inverse(const FourierArgs& a, float2* xb, float2* stage, const float2* tw,
                                            int j, int jj, int rb, const float2* slot) {
  using C = FCfg<N>;
  const int g = threadIdx.x / C::R2, t = threadIdx.x % C::R2;
  if (g >= C::GR) return;
  const int y = rb * C::GR + g;
  const int2 p = a.pos[j];
  const float2* orow = a.obj + (size_t)(p.x + y) * a.W + p.y;
  float2* xg = xb + g * C::XB;
  // c_j accumulator for this row; each thread owns the positions its pass 2
  // produces, so no synchronisation is needed.
  float2* cacc = stage + g * N;
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
    for (int k1 = 0; k1 < C::R1; ++k1) xg[k1 * C::R2 + (t ^ (k1 & (C::R2 - 1)))] = v[p1_index<N>(k1)];
    __syncwarp();
#pragma unroll
    for (int d = 0; d < C::D; ++d)
#pragma unroll
      for (int tt = 0; tt < C::R2; ++tt) v[d * C::R2 + tt] = xg[(t + C::R2 * d) * C::R2 + (tt ^ t)];
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

struct Pipe {                     // per-CTA bookkeeping of the shared-memory barriers
  uint32_t issued[kMaxStripBufs];  // TMA loads issued on barrier b (one per strip buffer)
  uint32_t done[kMaxStripBufs];    // TMA loads waited for
};

__device__ __forceinline__ void pipe_wait(Pipe& p, uint64_t* bars, int b, int* status) {
  mbar_wait_bounded(&bars[b], p.done[b] & 1u, status);
  p.done[b]++;
}

// ------------------------------------------------------------------ C task
// Strips of kStripW columns of every mode move between the row-major scratch
// and shared memory as 3-D TMA boxes (kStripW x N rows x M modes), laid out
// [mode][row][column] in shared memory.  The task's strips are double-buffered:
// the next strip's box and intensities load while the current one is
// transformed, and U goes back with a TMA store.  Column c of mode k is the
// stride-kStripW sequence at colbuf + k N kStripW + c; its exchange slots
// follow the in-place XOR pattern of the row transforms.
template <int N, bool INV>
__device__ __forceinline__ void strip_dft(float2* sb, int M, const float2* tw) {
  using C = FCfg<N>;
  constexpr int SW = kStripW;
  const int g = threadIdx.x / C::R2, t = threadIdx.x % C::R2;
  const int ncol = M * SW;
  for (int col0 = 0; col0 < ncol; col0 += C::GROUPS) {
    const int col = col0 + g;
    const bool act = col < ncol;
    const int k = act ? col / SW : 0, c = col % SW;
    float2* base = sb + k * N * SW + c;
    float2 v[C::R1];
    if (act) {
#pragma unroll
      for (int i = 0; i < C::R1; ++i) v[i] = base[(t + C::R2 * i) * SW];
      fft_pass1<N, INV>(v, t, tw);
    }
    __syncwarp();
    if (act) {
#pragma unroll
      for (int k1 = 0; k1 < C::R1; ++k1) base[(k1 * C::R2 + (t ^ (k1 & (C::R2 - 1)))) * SW] = v[p1_index<N>(k1)];
    }
    __syncwarp();
    if (act) {
#pragma unroll
      for (int d = 0; d < C::D; ++d)
#pragma unroll
        for (int tt = 0; tt < C::R2; ++tt) v[d * C::R2 + tt] = base[((t + C::R2 * d) * C::R2 + (tt ^ t)) * SW];
      fft_pass2<N, INV>(v);
    }
    __syncwarp();
    if (act) {
#pragma unroll
      for (int d = 0; d < C::D; ++d)
#pragma unroll
        for (int k2 = 0; k2 < C::R2; ++k2) base[(t + C::R2 * d + C::R1 * k2) * SW] = v[p2_index<N>(d, k2)];
    }
    __syncwarp();
  }
}

// Modulus projection of one strip, fused with the step to U (see the header):
// for every pixel of the strip, S = sum_k |X_k|^2, the scale s = sqrt(I) /
// (N sqrt(S)) (0 where S = 0) and X_k <- (beta s - 1/N^2) X_k; returns this
// thread's Fourier-error terms added to `ef`.  MM >= M bounds the unrolled
// mode loops so that the loads of all modes are in flight together.
template <int N, int MM>
__device__ __forceinline__ float modulus_strip(float2* sb, const float* ib, int M, float beta, float ef) {
  constexpr int SW = kStripW;
  const float invN = 1.f / (float)N;
  const float invN2 = invN * invN;
  for (int pq = threadIdx.x; pq < N * SW; pq += kThreads) {
    const int y = pq / SW, c = pq % SW;   // ib is [column][row]
    float S = 0.f;
#pragma unroll
    for (int k = 0; k < MM; ++k)
      if (k < M) S += cnorm(sb[k * N * SW + pq]);
    const float si_ = sqrtf(ib[c * N + y]);
    const float ss = sqrtf(S);
    const float sc = (S > 0.f) ? (si_ / ss) * invN : 0.f;
    const float dd = fmaf(ss, invN, -si_);
    ef = fmaf(dd, dd, ef);
    const float f = fmaf(beta, sc, -invN2);
#pragma unroll
    for (int k = 0; k < MM; ++k)
      if (k < M) sb[k * N * SW + pq] = cscale(sb[k * N * SW + pq], f);
  }
  return ef;
}

template <int N>
__device__ __forceinline__ double column_task(const FourierArgs& a, const CUtensorMap* tmap, float2* sbuf,
                                              float* ibuf, const float2* tw, uint64_t* bars, Pipe& pp, int j,
                                              int zview, int sg) {
  constexpr int SW = kStripW;
  const int M = a.M;
  const int tid = threadIdx.x;
  const float beta = a.beta;
  const int nbuf = a.strip_bufs;
  // strips loaded ahead of the one being transformed; with three buffers the
  // buffer a new load goes to was stored from one strip earlier, so its
  // store has had a whole strip's time to drain
  const int ahead = nbuf < 2 ? nbuf : 2;
  const uint32_t strip_elems = (uint32_t)M * N * SW;
  const uint32_t strip_bytes = strip_elems * (uint32_t)sizeof(float2);
  float ef = 0.f;  // this thread's few terms; the cross-thread sums are FP64
  auto issue = [&](int si) {  // strip si of the task into buffer si % nbuf (all threads)
    const int s = sg * a.SPG + si;
    const int b = si % nbuf;
    if (tid == 0) {
      mbar_arrive_expect_tx(&bars[b], strip_bytes);
      tma_load_3d(sbuf + (size_t)b * strip_elems, tmap, s * SW, 0, zview, &bars[b]);
    }
    pp.issued[b]++;
    const float* ist = a.istrip + ((size_t)j * a.NS + s) * (N * SW);
    for (int q = tid; q < (N * SW) / 4; q += kThreads) cp_async16(ibuf + b * (N * SW) + 4 * q, ist + 4 * q);
    cp_async_commit();
  };
  if (tid == 0) fence_proxy_async_global();
  issue(0);
  if (ahead > 1 && a.SPG > 1) issue(1);
  for (int si = 0; si < a.SPG; ++si) {
    const int s = sg * a.SPG + si;
    const int b = si % nbuf;
    float2* sb = sbuf + (size_t)b * strip_elems;
    const float* ib = ibuf + b * (N * SW);
    if (tid == 0) pipe_wait(pp, bars, b, a.status);
    else pp.done[b]++;
    __syncthreads();
    strip_dft<N, false>(sb, M, tw);
    if (ahead > 1 && si + 1 < a.SPG) cp_async_wait<1>(); else cp_async_wait<0>();
    __syncthreads();
    if (M <= 1) ef = modulus_strip<N, 1>(sb, ib, M, beta, ef);
    else if (M <= 2) ef = modulus_strip<N, 2>(sb, ib, M, beta, ef);
    else if (M <= 4) ef = modulus_strip<N, 4>(sb, ib, M, beta, ef);
    else if (M <= 8) ef = modulus_strip<N, 8>(sb, ib, M, beta, ef);
    else ef = modulus_strip<N, kMaxModes>(sb, ib, M, beta, ef);
    __syncthreads();
    strip_dft<N, true>(sb, M, tw);
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tma_store_3d(tmap, s * SW, 0, zview, sb);
      bulk_commit();
    }
    const int nxt = si + ahead;
    if (nxt < a.SPG) {
      // the buffer of strip nxt last held strip nxt - nbuf: wait until its
      // store has left shared memory
      if (tid == 0) {
        if (nbuf > ahead) bulk_wait_read<1>();
        else bulk_wait_read<0>();
      }
      __syncthreads();
      issue(nxt);
    }
  }
  return (double)ef;
}

template <int N>
__global__ void __launch_bounds__(kThreads, 2)
    k_fourier(const __grid_constant__ CUtensorMap tmap, const FourierArgs a) {
  using C = FCfg<N>;
  extern __shared__ unsigned char smem_raw[];
  // 128-byte aligned base (TMA boxes land at 128-byte aligned addresses)
  float2* tw = reinterpret_cast<float2*>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
  float2* work = tw + kTwBytes / sizeof(float2);
  // row tasks: exchange buffers, then two row buffers per transform (staged
  // psi and P rows of R; the object-source accumulator of I); column tasks:
  // the strip buffers, then their intensities
  float2* xb = work;
  float2* stage = work + C::GR * C::XB;
  float2* sbuf = work;
  float* ibuf = reinterpret_cast<float*>(work + (size_t)a.strip_bufs * a.M * N * kStripW);
  __shared__ __align__(8) uint64_t bars[kMaxStripBufs];
  __shared__ int s_task;
  __shared__ int s_skip;
  __shared__ double s_red[kThreads / 32];
  for (int i = threadIdx.x; i < N; i += kThreads) tw[i] = a.tw[i];
  if (threadIdx.x == 0) {
    for (int b = 0; b < kMaxStripBufs; ++b) mbar_init(&bars[b], 1);
    fence_mbar_init();
  }
  Pipe pp = {};

  int* disp = a.counters;
  int* doneR = a.counters + 1;
  int* doneC = doneR + a.nchunks;
  int* doneI = doneC + a.nchunks;
  int next = 0;
  if (threadIdx.x == 0) next = atomicAdd(disp, 1);
  int st_prev = 0;
  const size_t slot_elems = (size_t)a.B * a.M * N * N;

  for (;;) {
    if (threadIdx.x == 0) {
      s_task = next;
      if (next < a.total_tasks) next = atomicAdd(disp, 1);
    }
    __syncthreads();
    const int task = s_task;
    if (task >= a.total_tasks) break;

    // Decode (stage, kind, chunk, local index).  A CTA's tasks increase, so
    // the stage is the previous one or a later one: look at the next stage
    // before falling back to a binary search.
    int lo = st_prev;
    if (__ldg(a.stage_off + lo + 1) <= task) {
      ++lo;
      if (__ldg(a.stage_off + lo + 1) <= task) {
        int hi = a.nstages;
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (__ldg(a.stage_off + mid) <= task) lo = mid; else hi = mid;
        }
      }
    }
    const int st = lo;
    st_prev = lo;
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
      const int sl = c % a.nslot;
      float2* slot = a.scratch + (size_t)sl * slot_elems;
      if (kind == 0) {
        const int jj = local / a.RB, rb = local % a.RB;
        row_forward<N>(a, xb, stage, tw, c * a.B + jj, jj, rb, slot);
      } else if (kind == 1) {
        const int jj = local / a.CG, sg = local % a.CG;
        const int j = c * a.B + jj;
        double ef = column_task<N>(a, &tmap, sbuf, ibuf, tw, bars, pp, j, (sl * a.B + jj) * a.M, sg);
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
        row_inverse<N>(a, xb, stage, tw, c * a.B + jj, jj, rb, slot);
      }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      bulk_wait<0>();   // TMA stores of the task have landed
      __threadfence();
      atomicAdd((kind == 0 ? doneR : kind == 1 ? doneC : doneI) + c, 1);
    }
  }
  // Copies that a timed-out wait left in flight must land before the CTA exits.
  if (threadIdx.x == 0) {
    for (int b = 0; b < kMaxStripBufs; ++b)
      while (pp.done[b] < pp.issued[b]) pipe_wait(pp, bars, b, a.status);
    bulk_wait<0>();
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
static size_t smem_for(int M, int bufs) {
  using C = FCfg<N>;
  const size_t rows = (size_t)C::GR * (C::XB + 2 * N);
  const size_t cols = (size_t)bufs * M * N * kStripW + (size_t)bufs * N * kStripW / 2;
  return 128 + kTwBytes + sizeof(float2) * (rows > cols ? rows : cols);
}

size_t fourier_smem_bytes(int N, int M, int bufs) {
  switch (N) {
    case 16: return smem_for<16>(M, bufs);
    case 32: return smem_for<32>(M, bufs);
    case 64: return smem_for<64>(M, bufs);
    case 128: return smem_for<128>(M, bufs);
    case 256: return smem_for<256>(M, bufs);
    default: return 0;
  }
}

static const void* fourier_kernel(int N) {
  switch (N) {
    case 16: return (const void*)k_fourier<16>;
    case 32: return (const void*)k_fourier<32>;
    case 64: return (const void*)k_fourier<64>;
    case 128: return (const void*)k_fourier<128>;
    case 256: return (const void*)k_fourier<256>;
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

cudaError_t launch_fourier(const void* tmap, const FourierArgs& a, int grid, size_t smem, cudaStream_t s) {
  const CUtensorMap& m = *static_cast<const CUtensorMap*>(tmap);
  switch (a.N) {
    case 16: k_fourier<16><<<grid, kThreads, smem, s>>>(m, a); break;
    case 32: k_fourier<32><<<grid, kThreads, smem, s>>>(m, a); break;
    case 64: k_fourier<64><<<grid, kThreads, smem, s>>>(m, a); break;
    case 128: k_fourier<128><<<grid, kThreads, smem, s>>>(m, a); break;
    case 256: k_fourier<256><<<grid, kThreads, smem, s>>>(m, a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace dmk
