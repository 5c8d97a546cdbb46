// Cluster form of the Fourier step (Eq. 3 with the constrained transform F_c
// of Sec. II) for 64 x 64 and 128 x 128 frames and at most 8 modes.
//
// One thread-block cluster per view and one CTA per mode: CTA k keeps the
// whole frame of mode k in shared memory (32 or 128 KB of complex64), so both 1-D
// passes of each 2-D DFT run out of shared memory and no intermediate goes
// through global memory.  The two sums over the modes that couple the CTAs
// -- S = sum_k |X_k|^2 of the modulus projection and the object source
// c_j = sum_k conj(P_k) psi'_k of Eq. 5 -- are reduce-scatters over
// distributed shared memory: CTA r sums its 1/M of the pixels over the
// shared memory of every CTA of the cluster, in mode order.
//
// Per view j, in CTA k (mode k), with PO = P_k O(r_j + .):
//   1 rows:    Phi = 2 PO - psi (from global memory), forward row DFT
//   2 columns: forward column DFT X, |X|^2 into the norm buffer
//      [cluster barrier A]
//   3 pixels of this CTA: S from every CTA's norms, the factor
//      f = beta sqrt(I) / (N sqrt(S)) - 1/N^2 (0 - 1/N^2 where S = 0) pushed
//      into every CTA's norm buffer; the Fourier-error terms
//      [cluster barrier B]
//   4 columns: inverse column DFT of f X
//   5 rows:    inverse row DFT G, psi' = (2 - beta) PO + G to global memory,
//      conj(P_k) psi' into the frame
//      [cluster barrier C]
//   6 pixels of this CTA: c_j = sum_k conj(P_k) psi'_k
//      [cluster barrier D: the frames may be overwritten]
// With the unnormalised inverse, IDFT2(f X) = beta P_F(Phi) - Phi, where
// P_F is the modulus projection, so psi' = psi + beta (P_F(Phi) - PO) needs
// no second read of psi.
//
// Every CTA of a cluster runs the same views (j = cluster, cluster + number
// of clusters, ...), so all of them reach every cluster barrier; clusters
// never wait on one another.
#include <cuda.h>
#include <cuda_runtime.h>

#include "dm_fft.cuh"
#include "dm_kernels.h"
#include "dm_psi.cuh"
#include "dm_ptx.cuh"

namespace dmk {
namespace {

// Shape of the kernel for frame side N: a 128-point line is 16 values x 8
// lanes (two radix stages), a 64-point line 8 x 8; each 8-lane group takes
// two lines per pass (512 threads for N = 128, 256 for N = 64).
template <int N>
struct CShape {
  static constexpr int kT = N == 128 ? 512 : 256;          // threads per CTA
  static constexpr int kGroups = kT / 8;                    // 8-lane transform groups
  static constexpr int kR1 = FftShape<N>::R1;               // values per lane
  static constexpr int kD = kR1 / 8;                        // pass-2 transforms per lane
  static constexpr int kPix = N * N;
  static constexpr size_t kFrameBytes = sizeof(float2) * kPix;   // 128 or 32 KB
  static constexpr size_t kNormBytes = sizeof(float) * kPix;     // 64 or 16 KB
  static constexpr size_t kTwBytes = sizeof(float2) * N;         // W_N^(t k1), t < 8, k1 < R1
  static constexpr int kMinBlocks = N == 128 ? 1 : 4;            // CTAs per SM the registers allow
  static_assert(FftShape<N>::R2 == 8 && (kR1 == 16 || kR1 == 8), "8-lane lines of 64 or 128 points");
  static_assert(N == 2 * kGroups, "each group takes two lines per pass");
};

// Frame position (row r, column x) as a float2 index: N/16 blocks of 16
// columns, each [N rows][16 complex] with the row's 16-byte pairs permuted by
// pair ^= r & 7.  A half-warp then touches 16 distinct 8-byte bank pairs for
//   - 8 consecutive columns of rows r and r ^ 4 (row passes), and
//   - 8 rows with distinct r & 7 of columns c and c ^ 1 (column passes).
template <int N>
__device__ __forceinline__ int fidx(int r, int x) {
  return (x >> 4) * (N * 16) + (r << 4) + (((((x & 15) >> 1) ^ (r & 7)) << 1) | (x & 1));
}

// Norm-buffer position of pixel (row q, column x), in the strip order of the
// intensities (strip s = x / 2: [s][q][x & 1]), the 32-word halves of odd
// strips swapped so that the two strips of a column pass's half-warp fall on
// different banks.
template <int N>
__device__ __forceinline__ int nidx_strip(int p) {   // p: pixel in strip order
  const int s = p / (2 * N);
  return s * (2 * N) + ((p % (2 * N)) ^ ((s & 1) << 4));
}
template <int N>
__device__ __forceinline__ int nidx(int q, int x) { return nidx_strip<N>((x >> 1) * (2 * N) + (q << 1) + (x & 1)); }

// Exchange slot, along the transformed line, of pass-1 output k1 of lane t.
// For fixed k1 the 8 lanes write 8 consecutive slots; for fixed (k1 group,
// t) the 8 lanes reading k1 = t' + 8 d hit slots with distinct low 3 bits.
__device__ __forceinline__ int xslot(int k1, int t) { return k1 * 8 + (t ^ (k1 & 7)); }

// Row of group g in the row passes: groups 2m and 2m + 1 (one half-warp)
// get rows r and r ^ 4.
__device__ __forceinline__ int group_row(int g) { return (g & ~7) | ((g & 1) << 2) | ((g >> 1) & 3); }

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_index() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_count() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return r;
}
// The address in CTA `rank`'s shared memory that corresponds to the local
// shared address `a` (shared::cluster window).
__device__ __forceinline__ uint32_t dsmem_addr(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ float4 ld_dsmem4(uint32_t a) {
  float4 v;
  asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void st_dsmem4(uint32_t a, float4 v) {
  asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" :: "r"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
               : "memory");
}
// The modulus factor of one pixel from its intensity I and mode sum S:
// beta sqrt(I) / (N sqrt(S)) - 1/N^2 (-1/N^2 where S = 0); adds the pixel's
// Fourier-error term (sqrt(S)/N - sqrt(I))^2 to ef.  sqrt(I), sqrt(S) and
// their ratio come from two reciprocal square roots: the factor needs FP32
// relative accuracy, not correct rounding.
__device__ __forceinline__ float modulus_factor(float iv, float S, float beta, float invN, float invN2, float& ef) {
  const float ri = rsqrtf(iv), rs = rsqrtf(S);
  const float si_ = iv > 0.f ? iv * ri : 0.f;
  const float ss = S > 0.f ? S * rs : 0.f;
  const float sc = S > 0.f ? si_ * rs * invN : 0.f;
  const float dd = fmaf(ss, invN, -si_);
  ef = fmaf(dd, dd, ef);
  return fmaf(beta, sc, -invN2);
}
// All threads of all CTAs of the cluster; shared-memory writes before it are
// visible cluster-wide after it.
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// One N-point DFT along a line of the frame by the 8 lanes of a group:
// v[i] = x[t + 8 i] on entry; on return X[t + 8 d + R1 k2] sits at
// v[p2_index(d, k2)].  `at(pos)` is the frame index of line position pos.
// The line is overwritten by the exchange; the first __syncwarp makes sure
// every lane has read its inputs from the line first.
template <int N, bool INV, class At>
__device__ __forceinline__ void line_dft(float2 (&v)[CShape<N>::kR1], int t, const float2* tw, float2* F, At at) {
  using C = CShape<N>;
  fft_pass1<N, INV>(v, t, tw);
  __syncwarp();
#pragma unroll
  for (int k1 = 0; k1 < C::kR1; ++k1) F[at(xslot(k1, t))] = v[p1_index<N>(k1)];
  __syncwarp();
#pragma unroll
  for (int d = 0; d < C::kD; ++d)
#pragma unroll
    for (int tt = 0; tt < 8; ++tt) v[d * 8 + tt] = F[at(xslot(t + 8 * d, tt))];
  __syncwarp();
  fft_pass2<N, INV>(v);
}

// Line position of output (d, k2) of lane t after line_dft.
template <int N>
__device__ __forceinline__ int out_pos(int t, int d, int k2) { return t + 8 * d + CShape<N>::kR1 * k2; }

template <int N, class PsiT>
__global__ void __launch_bounds__(CShape<N>::kT, CShape<N>::kMinBlocks)
    k_fourier_cluster(const __grid_constant__ FourierArgs a) {
  using C = CShape<N>;
  constexpr int kCT = C::kT, kCGroups = C::kGroups, kCPix = C::kPix, kR1 = C::kR1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* F = reinterpret_cast<float2*>(smem_raw);
  float* NB = reinterpret_cast<float*>(smem_raw + C::kFrameBytes);
  float2* tw = reinterpret_cast<float2*>(smem_raw + C::kFrameBytes + C::kNormBytes);
  __shared__ double s_red[kCT / 32];

  const int tid = threadIdx.x, g = tid >> 3, t = tid & 7;
  const int M = a.M;
  const int r = (int)cluster_rank();         // this CTA's mode
  const float beta = a.beta, c2b = 2.f - beta;
  const float invN = 1.f / (float)N, invN2 = invN * invN;
  const uint32_t f_s = smem_u32(F), nb_s = smem_u32(NB);
  for (int i = tid; i < N; i += kCT) tw[i] = a.tw[i];
  __syncthreads();

  // this CTA's share of the pixels in steps 3 (strip order, in fours) and 6
  // (pairs in natural order)
  const int plo = 4 * (int)(((long long)r * (kCPix / 4)) / M), phi = 4 * (int)(((long long)(r + 1) * (kCPix / 4)) / M);
  const int qlo = (int)(((long long)r * (kCPix / 2)) / M), qhi = (int)(((long long)(r + 1) * (kCPix / 2)) / M);

  for (int j = (int)cluster_index(); j < a.J; j += (int)cluster_count()) {
    const int2 pos = a.pos[j];
    const PsiT* psi_k = static_cast<const PsiT*>(a.psi) + ((size_t)j * M + r) * kCPix;
    const float2* P_k = a.probe + (size_t)r * kCPix;

    // ---- 1: exit wave and forward row DFTs ----
#pragma unroll 1
    for (int rho = 0; rho < 2; ++rho) {
      const int y = group_row(g) + kCGroups * rho;
      const float2* prow = P_k + (size_t)y * N;
      const float2* orow = a.obj + (size_t)(pos.x + y) * a.W + pos.y;
      const PsiT* srow = psi_k + (size_t)y * N;
      float2 v[kR1];
#pragma unroll
      for (int i = 0; i < kR1; ++i) {
        const int x = t + 8 * i;
        const float2 po = cmul(__ldg(prow + x), __ldg(orow + x));
        const float2 s = psi_ldcs(srow + x);
        v[i] = make_float2(fmaf(2.f, po.x, -s.x), fmaf(2.f, po.y, -s.y));
      }
      line_dft<N, false>(v, t, tw, F, [&](int p) { return fidx<N>(y, p); });
#pragma unroll
      for (int d = 0; d < C::kD; ++d)
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) F[fidx<N>(y, out_pos<N>(t, d, k2))] = v[p2_index<N>(d, k2)];
    }
    __syncthreads();

    // ---- 2: forward column DFTs and |X|^2 ----
#pragma unroll 1
    for (int rho = 0; rho < 2; ++rho) {
      const int c = g + kCGroups * rho;
      float2 v[kR1];
#pragma unroll
      for (int i = 0; i < kR1; ++i) v[i] = F[fidx<N>(t + 8 * i, c)];
      line_dft<N, false>(v, t, tw, F, [&](int p) { return fidx<N>(p, c); });
#pragma unroll
      for (int d = 0; d < C::kD; ++d)
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) {
          const int q = out_pos<N>(t, d, k2);
          const float2 X = v[p2_index<N>(d, k2)];
          F[fidx<N>(q, c)] = X;
          NB[nidx<N>(q, c)] = cnorm(X);
        }
    }
    cluster_sync();   // A: every mode's norms are in place

    // ---- 3: modulus factors of this CTA's pixels, pushed to every CTA ----
    // four pixels per step: four consecutive strip-order pixels are four
    // consecutive floats of the norm buffer (its swizzle moves 16-float runs)
    float ef = 0.f;
    const float* inten = a.istrip + (size_t)j * kCPix;   // strip order, as p below
    for (int p = plo + 4 * tid; p < phi; p += 4 * kCT) {
      const uint32_t off = 4u * (uint32_t)nidx_strip<N>(p);
      float4 S = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int k = 0; k < M; ++k) {
        const float4 n = ld_dsmem4(dsmem_addr(nb_s + off, (uint32_t)k));
        S.x += n.x; S.y += n.y; S.z += n.z; S.w += n.w;
      }
      const float4 iv = __ldcs(reinterpret_cast<const float4*>(inten + p));
      float4 f;
      f.x = modulus_factor(iv.x, S.x, beta, invN, invN2, ef);
      f.y = modulus_factor(iv.y, S.y, beta, invN, invN2, ef);
      f.z = modulus_factor(iv.z, S.z, beta, invN, invN2, ef);
      f.w = modulus_factor(iv.w, S.w, beta, invN, invN2, ef);
      for (int k = 0; k < M; ++k) st_dsmem4(dsmem_addr(nb_s + off, (uint32_t)k), f);
    }
    {
      double e = (double)ef;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
      if ((tid & 31) == 0) s_red[tid >> 5] = e;
    }
    cluster_sync();   // B: every factor is in place (and this CTA's error partials)
    if (tid == 0) {
      double tot = 0.0;
      for (int i = 0; i < kCT / 32; ++i) tot += s_red[i];
      a.ef_part[(size_t)j * M + r] = tot;
    }

    // ---- 4: inverse column DFTs of f X ----
#pragma unroll 1
    for (int rho = 0; rho < 2; ++rho) {
      const int c = g + kCGroups * rho;
      float2 v[kR1];
#pragma unroll
      for (int i = 0; i < kR1; ++i) {
        const int q = t + 8 * i;
        v[i] = cscale(F[fidx<N>(q, c)], NB[nidx<N>(q, c)]);
      }
      line_dft<N, true>(v, t, tw, F, [&](int p) { return fidx<N>(p, c); });
#pragma unroll
      for (int d = 0; d < C::kD; ++d)
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) F[fidx<N>(out_pos<N>(t, d, k2), c)] = v[p2_index<N>(d, k2)];
    }
    __syncthreads();

    // ---- 5: inverse row DFTs, psi', conj(P_k) psi' ----
#pragma unroll 1
    for (int rho = 0; rho < 2; ++rho) {
      const int y = group_row(g) + kCGroups * rho;
      const float2* prow = P_k + (size_t)y * N;
      const float2* orow = a.obj + (size_t)(pos.x + y) * a.W + pos.y;
      PsiT* srow = static_cast<PsiT*>(a.psi) + ((size_t)j * M + r) * kCPix + (size_t)y * N;
      float2 v[kR1];
#pragma unroll
      for (int i = 0; i < kR1; ++i) v[i] = F[fidx<N>(y, t + 8 * i)];
      line_dft<N, true>(v, t, tw, F, [&](int p) { return fidx<N>(y, p); });
#pragma unroll
      for (int d = 0; d < C::kD; ++d)
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) {
          const int x = out_pos<N>(t, d, k2);
          const float2 pk = __ldg(prow + x);
          const float2 po = cmul(pk, __ldg(orow + x));
          const float2 g2 = v[p2_index<N>(d, k2)];
          const float2 pn = make_float2(fmaf(c2b, po.x, g2.x), fmaf(c2b, po.y, g2.y));
          psi_stcs(srow + x, pn);
          F[fidx<N>(y, x)] = cconjmul(pk, pn);
        }
    }
    cluster_sync();   // C: every mode's conj(P_k) psi'_k is in place

    // ---- 6: object source c_j of this CTA's pixels (two per thread) ----
    float2* cv = a.cview + (size_t)j * kCPix;
    for (int pp = qlo + tid; pp < qhi; pp += kCT) {
      const int px = 2 * pp, q = px / N, x = px & (N - 1);
      const uint32_t off = 8u * (uint32_t)fidx<N>(q, x);   // x even: the pair is one 16-byte chunk
      float4 acc = ld_dsmem4(dsmem_addr(f_s + off, 0));
      for (int k = 1; k < M; ++k) {
        const float4 u = ld_dsmem4(dsmem_addr(f_s + off, (uint32_t)k));
        const float2 lo = cadd(make_float2(acc.x, acc.y), make_float2(u.x, u.y));
        const float2 hi = cadd(make_float2(acc.z, acc.w), make_float2(u.z, u.w));
        acc = make_float4(lo.x, lo.y, hi.x, hi.y);
      }
      __stcs(reinterpret_cast<float4*>(cv + px), acc);
    }
    cluster_sync();   // D: no CTA reads this frame any more
  }
}

template <int N, class PsiT>
cudaError_t set_cluster_attrs() {
  return cudaFuncSetAttribute(k_fourier_cluster<N, PsiT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)fourier_cluster_smem_bytes(N));
}

template <int N>
cudaLaunchConfig_t cluster_config(int nclusters, int M, cudaStream_t s, cudaLaunchAttribute* at) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nclusters * M));
  cfg.blockDim = dim3(CShape<N>::kT);
  cfg.dynamicSmemBytes = fourier_cluster_smem_bytes(N);
  cfg.stream = s;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)M;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cfg;
}

template <int N>
int capacity(int M) {
  if (set_cluster_attrs<N, float2>() != cudaSuccess || set_cluster_attrs<N, __half2>() != cudaSuccess) return 0;
  cudaLaunchAttribute at[1];
  const cudaLaunchConfig_t cfg = cluster_config<N>(1, M, 0, at);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_fourier_cluster<N, float2>, &cfg) != cudaSuccess) return 0;
  return n;
}

template <int N>
cudaError_t launch(const FourierArgs& a, int nclusters, cudaStream_t s) {
  cudaLaunchAttribute at[1];
  const cudaLaunchConfig_t cfg = cluster_config<N>(nclusters, a.M, s, at);
  if (a.psi16) return cudaLaunchKernelEx(&cfg, k_fourier_cluster<N, __half2>, a);
  return cudaLaunchKernelEx(&cfg, k_fourier_cluster<N, float2>, a);
}

}  // namespace

bool fourier_cluster_shape(int N, int M) { return (N == 64 || N == 128) && M >= 1 && M <= kClusterMaxModes; }

size_t fourier_cluster_smem_bytes(int N) {
  if (N == 128) return CShape<128>::kFrameBytes + CShape<128>::kNormBytes + CShape<128>::kTwBytes;
  if (N == 64) return CShape<64>::kFrameBytes + CShape<64>::kNormBytes + CShape<64>::kTwBytes;
  return 0;
}

int fourier_cluster_capacity(int N, int M) {
  if (!fourier_cluster_shape(N, M)) return 0;
  return N == 128 ? capacity<128>(M) : capacity<64>(M);
}

cudaError_t launch_fourier_cluster(const FourierArgs& a, int nclusters, cudaStream_t s) {
  if (!fourier_cluster_shape(a.N, a.M) || nclusters < 1) return cudaErrorInvalidValue;
  return a.N == 128 ? launch<128>(a, nclusters, s) : launch<64>(a, nclusters, s);
}

}  // namespace dmk
