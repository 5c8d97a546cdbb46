// Cluster form of the Fourier step (Eq. 3 with the constrained transform F_c
// of Sec. II) for 128 x 128 frames and at most 8 modes.
//
// One thread-block cluster per view and one CTA per mode: CTA k keeps the
// whole frame of mode k in shared memory (128 KB of complex64), so both 1-D
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

constexpr int kCN = kClusterN;                 // frame side
constexpr int kCT = 512;                       // threads per CTA
constexpr int kCGroups = kCT / 8;              // 8-lane transform groups (64)
constexpr int kCPix = kCN * kCN;
static_assert(FftShape<kCN>::R1 == 16 && FftShape<kCN>::R2 == 8, "the layouts below assume 128 = 16 x 8");
static_assert(kCN == 2 * kCGroups, "each group takes two lines per pass");
constexpr size_t kFrameBytes = sizeof(float2) * kCPix;     // 128 KB
constexpr size_t kNormBytes = sizeof(float) * kCPix;       // 64 KB
constexpr size_t kTwCBytes = sizeof(float2) * kCN;         // W_128^(t k1), t < 8, k1 < 16

// Frame position (row r, column x) as a float2 index: 8 blocks of 16 columns,
// each [128 rows][16 complex] with the row's 16-byte pairs permuted by
// pair ^= r & 7.  A half-warp then touches 16 distinct 8-byte bank pairs for
//   - 8 consecutive columns of rows r and r ^ 4 (row passes), and
//   - 8 rows with distinct r & 7 of columns c and c ^ 1 (column passes).
__device__ __forceinline__ int fidx(int r, int x) {
  return ((x >> 4) << 11) + (r << 4) + (((((x & 15) >> 1) ^ (r & 7)) << 1) | (x & 1));
}

// Norm-buffer position of pixel (row q, column x), in the strip order of the
// intensities (strip s = x / 2: [s][q][x & 1]), the 32-word halves of odd
// strips swapped so that the two strips of a column pass's half-warp fall on
// different banks.
__device__ __forceinline__ int nidx_strip(int p) {   // p: pixel in strip order
  const int s = p >> 8;
  return (s << 8) + ((p & 255) ^ ((s & 1) << 4));
}
__device__ __forceinline__ int nidx(int q, int x) { return nidx_strip(((x >> 1) << 8) + (q << 1) + (x & 1)); }

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

// One 128-point DFT along a line of the frame by the 8 lanes of a group:
// v[i] = x[t + 8 i] on entry; on return X[t + 8 d + 16 k2] sits at
// v[p2_index(d, k2)].  `at(pos)` is the frame index of line position pos.
// The line is overwritten by the exchange; the first __syncwarp makes sure
// every lane has read its inputs from the line first.
template <bool INV, class At>
__device__ __forceinline__ void line_dft(float2 (&v)[16], int t, const float2* tw, float2* F, At at) {
  fft_pass1<kCN, INV>(v, t, tw);
  __syncwarp();
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) F[at(xslot(k1, t))] = v[p1_index<kCN>(k1)];
  __syncwarp();
#pragma unroll
  for (int d = 0; d < 2; ++d)
#pragma unroll
    for (int tt = 0; tt < 8; ++tt) v[d * 8 + tt] = F[at(xslot(t + 8 * d, tt))];
  __syncwarp();
  fft_pass2<kCN, INV>(v);
}

template <class PsiT>
__global__ void __launch_bounds__(kCT, 1) k_fourier_cluster(const __grid_constant__ FourierArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* F = reinterpret_cast<float2*>(smem_raw);
  float* NB = reinterpret_cast<float*>(smem_raw + kFrameBytes);
  float2* tw = reinterpret_cast<float2*>(smem_raw + kFrameBytes + kNormBytes);
  __shared__ double s_red[kCT / 32];

  const int tid = threadIdx.x, g = tid >> 3, t = tid & 7;
  const int M = a.M;
  const int r = (int)cluster_rank();         // this CTA's mode
  const float beta = a.beta, c2b = 2.f - beta;
  const float invN = 1.f / (float)kCN, invN2 = invN * invN;
  const uint32_t f_s = smem_u32(F), nb_s = smem_u32(NB);
  for (int i = tid; i < kCN; i += kCT) tw[i] = a.tw[i];
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
      const float2* prow = P_k + (size_t)y * kCN;
      const float2* orow = a.obj + (size_t)(pos.x + y) * a.W + pos.y;
      const PsiT* srow = psi_k + (size_t)y * kCN;
      float2 v[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int x = t + 8 * i;
        const float2 po = cmul(__ldg(prow + x), __ldg(orow + x));
        const float2 s = psi_ldcs(srow + x);
        v[i] = make_float2(fmaf(2.f, po.x, -s.x), fmaf(2.f, po.y, -s.y));
      }
      line_dft<false>(v, t, tw, F, [&](int p) { return fidx(y, p); });
#pragma unroll
      for (int d = 0; d < 2; ++d)
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) F[fidx(y, t + 8 * d + 16 * k2)] = v[p2_index<kCN>(d, k2)];
    }
    __syncthreads();

    // ---- 2: forward column DFTs and |X|^2 ----
#pragma unroll 1
    for (int rho = 0; rho < 2; ++rho) {
      const int c = g + kCGroups * rho;
      float2 v[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = F[fidx(t + 8 * i, c)];
      line_dft<false>(v, t, tw, F, [&](int p) { return fidx(p, c); });
#pragma unroll
      for (int d = 0; d < 2; ++d)
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) {
          const int q = t + 8 * d + 16 * k2;
          const float2 X = v[p2_index<kCN>(d, k2)];
          F[fidx(q, c)] = X;
          NB[nidx(q, c)] = cnorm(X);
        }
    }
    cluster_sync();   // A: every mode's norms are in place

    // ---- 3: modulus factors of this CTA's pixels, pushed to every CTA ----
    // four pixels per step: four consecutive strip-order pixels are four
    // consecutive floats of the norm buffer (its swizzle moves 16-float runs)
    float ef = 0.f;
    const float* inten = a.istrip + (size_t)j * kCPix;   // strip order, as p below
    for (int p = plo + 4 * tid; p < phi; p += 4 * kCT) {
      const uint32_t off = 4u * (uint32_t)nidx_strip(p);
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
      float2 v[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int q = t + 8 * i;
        v[i] = cscale(F[fidx(q, c)], NB[nidx(q, c)]);
      }
      line_dft<true>(v, t, tw, F, [&](int p) { return fidx(p, c); });
#pragma unroll
      for (int d = 0; d < 2; ++d)
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) F[fidx(t + 8 * d + 16 * k2, c)] = v[p2_index<kCN>(d, k2)];
    }
    __syncthreads();

    // ---- 5: inverse row DFTs, psi', conj(P_k) psi' ----
#pragma unroll 1
    for (int rho = 0; rho < 2; ++rho) {
      const int y = group_row(g) + kCGroups * rho;
      const float2* prow = P_k + (size_t)y * kCN;
      const float2* orow = a.obj + (size_t)(pos.x + y) * a.W + pos.y;
      PsiT* srow = static_cast<PsiT*>(a.psi) + ((size_t)j * M + r) * kCPix + (size_t)y * kCN;
      float2 v[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = F[fidx(y, t + 8 * i)];
      line_dft<true>(v, t, tw, F, [&](int p) { return fidx(y, p); });
#pragma unroll
      for (int d = 0; d < 2; ++d)
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) {
          const int x = t + 8 * d + 16 * k2;
          const float2 pk = __ldg(prow + x);
          const float2 po = cmul(pk, __ldg(orow + x));
          const float2 g2 = v[p2_index<kCN>(d, k2)];
          const float2 pn = make_float2(fmaf(c2b, po.x, g2.x), fmaf(c2b, po.y, g2.y));
          psi_stcs(srow + x, pn);
          F[fidx(y, x)] = cconjmul(pk, pn);
        }
    }
    cluster_sync();   // C: every mode's conj(P_k) psi'_k is in place

    // ---- 6: object source c_j of this CTA's pixels (two per thread) ----
    float2* cv = a.cview + (size_t)j * kCPix;
    for (int pp = qlo + tid; pp < qhi; pp += kCT) {
      const int px = 2 * pp, q = px >> 7, x = px & (kCN - 1);
      const uint32_t off = 8u * (uint32_t)fidx(q, x);   // x even: the pair is one 16-byte chunk
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

template <class PsiT>
cudaError_t set_cluster_attrs() {
  return cudaFuncSetAttribute(k_fourier_cluster<PsiT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)fourier_cluster_smem_bytes());
}

template <class PsiT>
cudaLaunchConfig_t cluster_config(int nclusters, int M, cudaStream_t s, cudaLaunchAttribute* at) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nclusters * M));
  cfg.blockDim = dim3(kCT);
  cfg.dynamicSmemBytes = fourier_cluster_smem_bytes();
  cfg.stream = s;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)M;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cfg;
}

}  // namespace

size_t fourier_cluster_smem_bytes() { return kFrameBytes + kNormBytes + kTwCBytes; }

int fourier_cluster_capacity(int M) {
  if (M < 1 || M > kClusterMaxModes) return 0;
  if (set_cluster_attrs<float2>() != cudaSuccess || set_cluster_attrs<__half2>() != cudaSuccess) return 0;
  cudaLaunchAttribute at[1];
  const cudaLaunchConfig_t cfg = cluster_config<float2>(1, M, 0, at);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_fourier_cluster<float2>, &cfg) != cudaSuccess) return 0;
  return n;
}

cudaError_t launch_fourier_cluster(const FourierArgs& a, int nclusters, cudaStream_t s) {
  if (a.N != kCN || a.M < 1 || a.M > kClusterMaxModes || nclusters < 1) return cudaErrorInvalidValue;
  cudaLaunchAttribute at[1];
  const cudaLaunchConfig_t cfg = cluster_config<float2>(nclusters, a.M, s, at);
  if (a.psi16) return cudaLaunchKernelEx(&cfg, k_fourier_cluster<__half2>, a);
  return cudaLaunchKernelEx(&cfg, k_fourier_cluster<float2>, a);
}

}  // namespace dmk
