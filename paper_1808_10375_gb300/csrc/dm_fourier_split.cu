// Fourier step of the difference map (Eq. 3 with the constrained transform
// F_c of Sec. II) for 256 x 256 frames with 8 probe modes, in the split-
// column form: the 256-point column DFT is split into two radix-16 stages,
// the first taken by the row tasks and the second by the column tasks.
//
// With rows y = n1 + 16 n2 and spectrum rows q = k1 + 16 k2 (n1, n2, k1, k2
// in [0, 16)) and T the row DFT of Phi = 2 P O - psi,
//   Y[k1][n1]  = W^(n1 k1) sum_n2 T[n1 + 16 n2] W16^(n2 k1)        (R task)
//   X[k1 + 16 k2] = sum_n1 Y[k1][n1] W16^(n1 k2)                     (C task)
// (W = exp(-2 pi i / 256), W16 = W^16), which is the unnormalised column
// DFT.  The C task scales X by f = beta sqrt(I) / (N sqrt(S)) - 1/N^2 with
// S = sum_k |X_k|^2 (the modulus projection of F_c folded with the psi
// update, as in the strip form) and takes the inverse of its own stage,
//   Z[k1][n1] = sum_k2 f X[k1 + 16 k2] W16^(-n1 k2),
// and the I task the inverse of the first,
//   U[n1 + 16 n2] = sum_k1 W16^(-n2 k1) W^(-n1 k1) Z[k1][n1],
// before the inverse row DFT and psi' = (2 - beta) P O + IDFT_rows(U).
//
// Why: in the strip form every column task moves 2-column strips (16-byte
// rows) and needs block barriers around the mode sum S.  Here a column-task
// item is the 16 values n1 of 16 columns and 8 modes for one k1: a 16 KB TMA
// box of 128-byte rows.  Each thread owns one (column, mode) pair and does
// its 16-point DFT in registers; the 8 modes of a column sit in 8 lanes of
// one warp, so S comes from warp shuffles and no block barrier is needed.
//
// Scratch layout of a view: [k1][n1][mode][column] (rows of 256 complex
// values).  Task kinds and counts per view: R (16, one per n1), C (16, one
// per k1: 16 items of 16 columns), I (16, one per n1).  The scheduling
// (chunks, stages, bounded waits) is the strip form's, with completion
// counters per view instead of per chunk.
#include <cuda.h>
#include <cuda_runtime.h>

#include "dm_fft.cuh"
#include "dm_kernels.h"
#include "dm_psi.cuh"
#include "dm_ptx.cuh"

#include <algorithm>

namespace dmk {

namespace {

constexpr int kN = kSplitN;             // frame side
constexpr int kM = kSplitModes;         // modes (one lane per mode in the column task)
constexpr int kR = 16;                  // radix of each stage (N = 16 x 16)
constexpr int kXS = kR * (kR + 1);      // padded exchange buffer of one row transform (values)
constexpr int kItemBytes = 16 * kR * kM * 8;   // 16 columns x 16 n1 x 8 modes of complex64
constexpr int kIBoxFloats = 16 * 16;           // intensities of one item
constexpr int kItemsPerLane = 8;               // items of a column task per item lane (2 lanes)
static_assert(kN == kR * kR && kM == 8, "the split form is written for 256 x 256 frames and 8 modes");

// Row buffers of the row tasks, per group g of 16 lanes (row n1 + 16 g): the
// padded exchange buffer, then two plain rows.
__device__ __forceinline__ float2* sp_xbuf(float2* stage, int g) { return stage + g * kXS; }
__device__ __forceinline__ float2* sp_row(float2* stage, int g, int i) {
  return stage + kR * kXS + (i * kR + g) * kN;
}

// Scratch row of (view jj of the slot, k1, n1, mode k).
__device__ __forceinline__ size_t sp_row_index(int jj, int k1, int n1, int k) {
  return (((size_t)jj * kR + k1) * kR + n1) * kM + k;
}

// ------------------------------------------------------------------ R task
// Rows y = n1 + 16 g: exit wave, row DFT (as in the strip form), then the
// first stage of the column DFT over the 16 rows of the task.  The row of T
// goes to the group's exchange buffer in natural order; after a block
// barrier thread c reads column c of the 16 rows, transforms it over n2,
// applies W^(n1 k1) and stores Y[k1][n1][k][c].  Staged copies per group:
// A psi of the next mode (a whole mode ahead), B the probe row (then the
// exchange, then the row of T; the next probe row is requested once the
// column reads are done), O the object row.
template <class PsiT>
__device__ __forceinline__ void split_row_forward(const FourierArgs& a, float2* stage, const float2* tw, int j,
                                                  int jj, int n1, float2* slot) {
  const int g = threadIdx.x / kR, t = threadIdx.x % kR, c = threadIdx.x;
  const int y = n1 + kR * g;
  const int2 p = a.pos[j];
  const float2* orow = a.obj + (size_t)(p.x + y) * a.W + p.y;
  float2* srow_s = sp_row(stage, g, 0);
  float2* xg = sp_xbuf(stage, g);
  float2* orow_s = sp_row(stage, g, 1);
  const uint64_t pol_first = l2_policy_evict_first(), pol_last = l2_policy_evict_last();
  auto issue_psi = [&](int k) {
    constexpr int kChunks = kN * (int)sizeof(PsiT) / 16;
    const char* src = reinterpret_cast<const char*>(static_cast<const PsiT*>(a.psi) + (((size_t)j * kM + k) * kN + y) * kN);
    char* dst = reinterpret_cast<char*>(srow_s);
    for (int q = t; q < kChunks; q += kR) cp_async16_hint(dst + 16 * q, src + 16 * q, pol_first);
  };
  auto issue_p = [&](int k) {
    const float2* src = a.probe + ((size_t)k * kN + y) * kN;
    for (int q = t; q < kN / 2; q += kR) cp_async16_hint(xg + 2 * q, src + 2 * q, pol_last);
  };
  const PsiT* srow_t = reinterpret_cast<const PsiT*>(srow_s);
  for (int x = t; x < kN; x += kR) cp_async8(orow_s + x, orow + x);
  issue_psi(0);
  issue_p(0);
  cp_async_commit();
  for (int k = 0; k < kM; ++k) {
    cp_async_wait<0>();
    __syncwarp();
    float2 v[kR];
#pragma unroll
    for (int i = 0; i < kR; ++i) {
      const int x = t + kR * i;
      const float2 po = cmul(xg[x], orow_s[x]);
      const float2 s = psi_ld(srow_t + x);
      v[i] = make_float2(fmaf(2.f, po.x, -s.x), fmaf(2.f, po.y, -s.y));
    }
    __syncwarp();
    const bool more = k + 1 < kM;
    if (more) { issue_psi(k + 1); cp_async_commit(); }
    fft_pass1<kN, false>(v, t, tw);
#pragma unroll
    for (int k1 = 0; k1 < kR; ++k1) xg[k1 * (kR + 1) + t] = v[p1_index<kN>(k1)];
    __syncwarp();
#pragma unroll
    for (int tt = 0; tt < kR; ++tt) v[tt] = xg[t * (kR + 1) + tt];
    __syncwarp();
    fft_pass2<kN, false>(v);
    // the row of T, natural order: T[y][t + 16 k2]
#pragma unroll
    for (int k2 = 0; k2 < kR; ++k2) xg[t + kR * k2] = v[p2_index<kN>(0, k2)];
    __syncthreads();
    float2 w[kR];
#pragma unroll
    for (int n2 = 0; n2 < kR; ++n2) w[n2] = sp_xbuf(stage, n2)[c];
    __syncthreads();   // every column is read: the buffers take the next probe rows
    if (more) { issue_p(k + 1); cp_async_commit(); }
    dft_reg<kR, false>(w);
    float2* col = slot + sp_row_index(jj, 0, n1, k) * kN + c;
#pragma unroll
    for (int k1 = 0; k1 < kR; ++k1) {
      float2 yv = w[out_index<kR>(k1)];
      if (k1 > 0) yv = cmul(yv, tw[k1 * kR + n1]);   // W^(n1 k1)
      st_cg_hint(col + (size_t)k1 * kR * kM * kN, yv, pol_last);
    }
  }
}

// ------------------------------------------------------------------ I task
// Thread c holds Z[k1][n1][k][c] for every k1 (loaded a whole mode ahead),
// applies W^(-n1 k1) and the inverse DFT over k1, which gives U of rows n1 +
// 16 n2 in column c; these go to the groups' exchange buffers (row n2 to
// group n2) and, after a block barrier, every group takes the inverse row
// DFT of its row and forms psi' and the object source as in the strip form.
// Staged per group: B the probe row of the mode, O the object row.
template <class PsiT>
__device__ __forceinline__ void split_row_inverse(const FourierArgs& a, float2* stage, const float2* tw, int j,
                                                  int jj, int n1, const float2* slot) {
  const int g = threadIdx.x / kR, t = threadIdx.x % kR, c = threadIdx.x;
  const int y = n1 + kR * g;
  const int2 p = a.pos[j];
  const float2* orow = a.obj + (size_t)(p.x + y) * a.W + p.y;
  float2* xg = sp_xbuf(stage, g);
  float2* prow_s = sp_row(stage, g, 0);
  float2* orow_s = sp_row(stage, g, 1);
  const float c2b = 2.f - a.beta;
  const uint64_t pol_last = l2_policy_evict_last();
  auto issue_p = [&](int k) {
    const float2* src = a.probe + ((size_t)k * kN + y) * kN;
    for (int q = t; q < kN / 2; q += kR) cp_async16_hint(prow_s + 2 * q, src + 2 * q, pol_last);
    cp_async_commit();
  };
  const float2* z0 = slot + sp_row_index(jj, 0, n1, 0) * kN + c;   // Z[k1 = 0][n1][mode 0][c]
  constexpr size_t kZk1 = (size_t)kR * kM * kN;                   // elements between consecutive k1
  float2 w[kR];
#pragma unroll
  for (int k1 = 0; k1 < kR; ++k1) w[k1] = __ldcg(z0 + k1 * kZk1);
  for (int x = t; x < kN; x += kR) cp_async8(orow_s + x, orow + x);
  issue_p(0);
  float2 cacc[kR];
  for (int k = 0; k < kM; ++k) {
#pragma unroll
    for (int k1 = 1; k1 < kR; ++k1) w[k1] = ctw<true>(w[k1], tw[k1 * kR + n1]);   // W^(-n1 k1)
    dft_reg<kR, true>(w);
#pragma unroll
    for (int n2 = 0; n2 < kR; ++n2) sp_xbuf(stage, n2)[c] = w[out_index<kR>(n2)];
    const bool more = k + 1 < kM;
    if (more) {
#pragma unroll
      for (int k1 = 0; k1 < kR; ++k1) w[k1] = __ldcg(z0 + (size_t)(k + 1) * kN + k1 * kZk1);
    }
    __syncthreads();
    // every read of this (n1, mode) is done: drop its 16 scratch rows from L2
    // unwritten (thread c: row k1 = c / 16, 128-byte line c % 16)
    l2_discard128(z0 - c + (size_t)k * kN + (size_t)(c / kR) * kZk1 + (c % kR) * 16);
    float2 v[kR];
#pragma unroll
    for (int i = 0; i < kR; ++i) v[i] = xg[t + kR * i];
    __syncwarp();
    fft_pass1<kN, true>(v, t, tw);
#pragma unroll
    for (int k1 = 0; k1 < kR; ++k1) xg[k1 * (kR + 1) + t] = v[p1_index<kN>(k1)];
    __syncwarp();
#pragma unroll
    for (int tt = 0; tt < kR; ++tt) v[tt] = xg[t * (kR + 1) + tt];
    __syncthreads();   // every group has read its row: the buffers take the next mode's columns
    fft_pass2<kN, true>(v);
    cp_async_wait<0>();   // P of this mode (and the object row)
    __syncwarp();
    PsiT* srow = static_cast<PsiT*>(a.psi) + (((size_t)j * kM + k) * kN + y) * kN;
#pragma unroll
    for (int k2 = 0; k2 < kR; ++k2) {
      const int x = t + kR * k2;
      const float2 pk = prow_s[x];
      const float2 po = cmul(pk, orow_s[x]);
      const float2 g2 = v[p2_index<kN>(0, k2)];
      const float2 pn = make_float2(fmaf(c2b, po.x, g2.x), fmaf(c2b, po.y, g2.y));
      psi_stcs(srow + x, pn);
      const float2 cn = cconjmul(pk, pn);
      cacc[k2] = k == 0 ? cn : cadd(cacc[k2], cn);
    }
    __syncwarp();
    if (more) issue_p(k + 1);
  }
  float2* crow = a.cview + ((size_t)j * kN + y) * kN;
#pragma unroll
  for (int k2 = 0; k2 < kR; ++k2) __stcs(crow + t + kR * k2, cacc[k2]);
}

// ------------------------------------------------------------------ C task
// The 16 items of (view, k1) go to two item lanes of four warps, item xb to
// lane xb % 2, each lane streaming its items through a ring of kSplitBufs
// buffers.  Thread (column c, mode m) of a lane: warp c / 4, lane m + 8 (c %
// 4).  The box is stored with the 128-byte swizzle (16-byte chunk ^ row % 8,
// and a box row is (n1, m)), so the 16 lanes of a half-warp, which read one
// chunk of 8 different modes, hit 16 different bank pairs.
struct SplitPipe {
  uint32_t issued[kSplitBufs];   // loads issued on buffer b of this thread's lane
  uint32_t done[kSplitBufs];     // loads waited for
};

__device__ __forceinline__ void split_wait(SplitPipe& p, uint64_t* bars, int b, int* status) {
  const uint32_t par = p.done[b] & 1u;
  if ((threadIdx.x & 31) == 0) mbar_wait_bounded(&bars[b], par, status);
  __syncwarp();
  (void)mbar_try_wait_parity(&bars[b], par);
  p.done[b]++;
}

// Sum over the 8 mode lanes (lane bits 0-2) of s[0..16), scattered: lane m
// returns the sums for k2 = 2m and 2m + 1.
__device__ __forceinline__ void mode_sum_scatter(const float (&s)[16], int m, float (&o)[2]) {
  const bool h1 = m & 4, h2 = m & 2, h3 = m & 1;
  float s8[8], s4[4];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float send = h1 ? s[i] : s[i + 8], keep = h1 ? s[i + 8] : s[i];
    s8[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float send = h2 ? s8[i] : s8[i + 4], keep = h2 ? s8[i + 4] : s8[i];
    s4[i] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float send = h3 ? s4[i] : s4[i + 2], keep = h3 ? s4[i + 2] : s4[i];
    o[i] = keep + __shfl_xor_sync(0xffffffffu, send, 1);
  }
}

// Inverse of the scatter's placement: lane m holds f for k2 = 2m, 2m + 1;
// every lane returns all 16.
__device__ __forceinline__ void mode_gather(const float (&f2)[2], int m, float (&f)[16]) {
  const bool h1 = m & 4, h2 = m & 2, h3 = m & 1;
  float f4[4], f8[8];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float r = __shfl_xor_sync(0xffffffffu, f2[i], 1);
    f4[i] = h3 ? r : f2[i];
    f4[i + 2] = h3 ? f2[i] : r;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float r = __shfl_xor_sync(0xffffffffu, f4[i], 2);
    f8[i] = h2 ? r : f4[i];
    f8[i + 4] = h2 ? f4[i] : r;
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float r = __shfl_xor_sync(0xffffffffu, f8[i], 4);
    f[i] = h1 ? r : f8[i];
    f[i + 8] = h1 ? f8[i] : r;
  }
}

// Returns this thread's Fourier-error terms (sqrt(S)/N - sqrt(I))^2.
__device__ __forceinline__ float split_column_task(const FourierArgs& a, const CUtensorMap* tmS,
                                                   const CUtensorMap* tmI, unsigned char* cbase, uint64_t* bars,
                                                   SplitPipe& pp, int j, int sl, int jj, int k1) {
  const int tid = threadIdx.x, L = tid >> 7, ti = tid & 127;
  const int lane = tid & 31, m = lane & 7, c = 4 * (ti >> 5) + (lane >> 3);
  const bool issuer = ti == 0;
  uint64_t* lb = bars + L * kSplitBufs;
  unsigned char* dbuf = cbase + (size_t)L * kSplitBufs * kItemBytes;
  float* ibox = reinterpret_cast<float*>(cbase + (size_t)2 * kSplitBufs * kItemBytes) + L * kSplitBufs * kIBoxFloats;
  const int row0 = ((sl * a.B + jj) * kR + k1) * kR * kM;   // scratch row of (n1 = 0, mode 0)
  const int irow0 = (j * kR + k1) * kN;                     // intensity row of column 0
  const float beta = a.beta;
  const float invN = 1.f / (float)kN, invN2 = invN * invN;
  const uint64_t pol_first = l2_policy_evict_first(), pol_last = l2_policy_evict_last();
  auto issue = [&](int i) {   // item i of the lane (columns 16 xb .. 16 xb + 15) into buffer i % kSplitBufs
    const int b = i % kSplitBufs, xb = L + 2 * i;
    if (issuer) {
      mbar_arrive_expect_tx(&lb[b], (uint32_t)(kItemBytes + kIBoxFloats * sizeof(float)));
      tma_load_2d_hint(dbuf + (size_t)b * kItemBytes, tmS, 16 * xb, row0, &lb[b], pol_last);
      tma_load_2d_hint(ibox + b * kIBoxFloats, tmI, 0, irow0 + 16 * xb, &lb[b], pol_first);
    }
    pp.issued[b]++;
  };
  if (issuer) fence_proxy_async_global();   // the row tasks' stores are visible to the TMA loads
#pragma unroll 1
  for (int i = 0; i < kSplitBufs && i < kItemsPerLane; ++i) issue(i);
  // byte offset of (n1 = 0, m, c) in a swizzled box: row m, chunk (c / 2) ^ m
  const int off = m * 128 + ((((c >> 1) ^ m) & 7) << 4) + ((c & 1) << 3);
  float ef = 0.f;
#pragma unroll 1
  for (int i = 0; i < kItemsPerLane; ++i) {
    const int b = i % kSplitBufs, xb = L + 2 * i;
    split_wait(pp, lb, b, a.status);
    unsigned char* d = dbuf + (size_t)b * kItemBytes;
    float2 v[kR];
#pragma unroll
    for (int n1 = 0; n1 < kR; ++n1) v[n1] = *reinterpret_cast<const float2*>(d + n1 * 1024 + off);
    dft_reg<kR, false>(v);   // X[k1 + 16 k2] at v[out_index(k2)]
    float s[16];
#pragma unroll
    for (int k2 = 0; k2 < kR; ++k2) s[k2] = cnorm(v[out_index<kR>(k2)]);
    float S2[2], f2[2];
    mode_sum_scatter(s, m, S2);
    const float2 iv = *reinterpret_cast<const float2*>(ibox + b * kIBoxFloats + c * 16 + 2 * m);
    const float I2[2] = {iv.x, iv.y};
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      // sqrt(I), sqrt(S) and sqrt(I)/sqrt(S) from two reciprocal square roots
      const float I = I2[q], S = S2[q];
      const float ri = rsqrtf(I), rs = rsqrtf(S);
      const float si = I > 0.f ? I * ri : 0.f;
      const float ss = S > 0.f ? S * rs : 0.f;
      const float sc = S > 0.f ? si * rs * invN : 0.f;
      const float dd = fmaf(ss, invN, -si);
      ef = fmaf(dd, dd, ef);
      f2[q] = fmaf(beta, sc, -invN2);
    }
    float f[16];
    mode_gather(f2, m, f);
    float2 u[kR];   // the scaled spectrum in natural k2 order (a renaming, no instructions)
#pragma unroll
    for (int k2 = 0; k2 < kR; ++k2) u[k2] = cscale(v[out_index<kR>(k2)], f[k2]);
    dft_reg<kR, true>(u);    // Z[k1][n1] at u[out_index(n1)]
#pragma unroll
    for (int n1 = 0; n1 < kR; ++n1) *reinterpret_cast<float2*>(d + n1 * 1024 + off) = u[out_index<kR>(n1)];
    fence_proxy_async_smem();
    named_bar_sync(1 + L, 128);   // the item is written (and every read of the buffer is done)
    if (issuer) {
      tma_store_2d_hint(tmS, 16 * xb, row0, d, pol_last);
      bulk_commit();
      if (i + kSplitBufs < kItemsPerLane) bulk_wait_read<0>();   // the buffer takes item i + kSplitBufs
    }
    if (i + kSplitBufs < kItemsPerLane) issue(i + kSplitBufs);
  }
  if (issuer) bulk_wait<0>();   // the lane's stores are complete before the task is published
  return ef;
}

}  // namespace

template <class PsiT>
__global__ void __launch_bounds__(kThreads, 2)
    k_fourier_split(const __grid_constant__ CUtensorMap tmS, const __grid_constant__ CUtensorMap tmI,
                    const FourierArgs a) {
  extern __shared__ unsigned char smem_raw[];
  // 1024-byte aligned base: the swizzled TMA boxes need it
  unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  float2* tw = reinterpret_cast<float2*>(base);
  unsigned char* work = base + kTwBytes;
  float2* stage = reinterpret_cast<float2*>(work);
  __shared__ __align__(8) uint64_t bars[2 * kSplitBufs];
  __shared__ int s_task;
  __shared__ int s_skip;
  __shared__ double s_red[kThreads / 32];
  for (int i = threadIdx.x; i < kN; i += kThreads) tw[i] = a.tw[i];
  if (threadIdx.x == 0) {
    for (int b = 0; b < 2 * kSplitBufs; ++b) mbar_init(&bars[b], 1);
    fence_mbar_init();
  }
  SplitPipe pp = {};

  // per-view completion counters (a column task waits for the row tasks of
  // its own view only, and so on), so that a task's wait does not extend to
  // the slowest task of its whole chunk
  int* disp = a.counters;
  int* doneR = a.counters + 1;
  int* doneC = doneR + a.J;
  int* doneI = doneC + a.J;
  int next = 0;
  if (threadIdx.x == 0) next = atomicAdd(disp, 1);
  int st_prev = 0;
  const size_t slot_elems = (size_t)a.B * kM * kN * kN;

  for (;;) {
    if (threadIdx.x == 0) {
      s_task = next;
      if (next < a.total_tasks) next = atomicAdd(disp, 1);
    }
    __syncthreads();
    const int task = s_task;
    if (task >= a.total_tasks) break;

    // Decode (stage, kind, chunk, local index) as in the strip form.
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
    int kind = -1, ch = 0;
    if (st < a.nchunks) {
      const int nv = min(a.B, a.J - st * a.B);
      if (local < nv * a.RB) { kind = 0; ch = st; } else local -= nv * a.RB;
    }
    if (kind < 0) {
      const int cc = st - a.lag;
      if (cc >= 0 && cc < a.nchunks) {
        const int nv = min(a.B, a.J - cc * a.B);
        if (local < nv * a.CG) { kind = 1; ch = cc; } else local -= nv * a.CG;
      }
    }
    if (kind < 0) { kind = 2; ch = st - 2 * a.lag; }

    const int jj = local / kR, r = local % kR;   // RB = CG = 16
    const int j = ch * a.B + jj;
    if (threadIdx.x == 0) {
      bool ok = true;
      if (kind == 0) {
        // the slot's area of this view was last used by view j - nslot B
        if (ch >= a.nslot) ok = spin_wait_geq(doneI + (j - a.nslot * a.B), a.RB, a.status);
      } else if (kind == 1) {
        ok = spin_wait_geq(doneR + j, a.RB, a.status);
      } else {
        ok = spin_wait_geq(doneC + j, a.CG, a.status);
      }
      s_skip = ok ? 0 : 1;
    }
    __syncthreads();

    if (!s_skip) {
      const int sl = ch % a.nslot;
      float2* slot = a.scratch + (size_t)sl * slot_elems;
      if (kind == 0) {
        split_row_forward<PsiT>(a, stage, tw, j, jj, r, slot);
      } else if (kind == 1) {
        double ef = split_column_task(a, &tmS, &tmI, work, bars, pp, j, sl, jj, r);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ef += __shfl_xor_sync(0xffffffffu, ef, o);
        if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = ef;
        __syncthreads();
        if (threadIdx.x == 0) {
          double tot = 0.0;
          for (int i = 0; i < kThreads / 32; ++i) tot += s_red[i];
          a.ef_part[(size_t)j * a.CG + r] = tot;
        }
      } else {
        split_row_inverse<PsiT>(a, stage, tw, j, jj, r, slot);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      bulk_wait<0>();
      __threadfence();
      atomicAdd((kind == 0 ? doneR : kind == 1 ? doneC : doneI) + j, 1);
    }
  }
  // Copies that a timed-out wait left in flight must land before the CTA exits.
  if ((threadIdx.x & 127) == 0) {
    uint64_t* lb = bars + (threadIdx.x >> 7) * kSplitBufs;
    for (int b = 0; b < kSplitBufs; ++b)
      while (pp.done[b] < pp.issued[b]) {
        mbar_wait_bounded(&lb[b], pp.done[b] & 1u, a.status);
        pp.done[b]++;
      }
    bulk_wait<0>();
  }
}

size_t fourier_split_smem_bytes() {
  static_assert((size_t)kR * kXS * 8 + (size_t)2 * kR * kN * 8 <=
                    (size_t)2 * kSplitBufs * (kItemBytes + kIBoxFloats * 4),
                "the row tasks' buffers fit in the column tasks' area");
  return 1024 + kTwBytes + (size_t)2 * kSplitBufs * (kItemBytes + kIBoxFloats * sizeof(float));
}

static const void* split_kernel(bool half) {
  return half ? (const void*)k_fourier_split<__half2> : (const void*)k_fourier_split<float2>;
}

int fourier_split_occupancy(size_t smem) {
  int best = -1;
  for (bool half : {false, true}) {
    const void* f = split_kernel(half);
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - 1024) != cudaSuccess) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, kThreads, smem) != cudaSuccess) return 0;
    best = best < 0 ? nb : (nb < best ? nb : best);
  }
  return best;
}

cudaError_t launch_fourier_split(const void* tmaps, const FourierArgs& a, int grid, size_t smem, cudaStream_t s) {
  const CUtensorMap* m = static_cast<const CUtensorMap*>(tmaps);
  if (a.N != kN || a.M != kM || a.psi_part) return cudaErrorInvalidValue;
  if (a.psi16) k_fourier_split<__half2><<<grid, kThreads, smem, s>>>(m[0], m[1], a);
  else k_fourier_split<float2><<<grid, kThreads, smem, s>>>(m[0], m[1], a);
  return cudaGetLastError();
}

// Intensities of the split form: isplit[j][k1][x][k2] = I[j][k1 + 16 k2][x],
// so that one column-task item's 16 columns x 16 rows k2 are one TMA box.
__global__ void __launch_bounds__(kThreads) k_intensity_split(float* isplit, const float* inten, int J) {
  const size_t tot = (size_t)J * kN * kN;
  for (size_t i = (size_t)blockIdx.x * kThreads + threadIdx.x; i < tot; i += (size_t)gridDim.x * kThreads) {
    const size_t jv = i / (kN * kN);
    const int r = (int)(i % (kN * kN)), yq = r / kN, x = r % kN;
    const int k1 = yq % kR, k2 = yq / kR;
    isplit[((jv * kR + k1) * kN + x) * kR + k2] = inten[i];
  }
}

cudaError_t launch_intensity_split(float* isplit, const float* inten, int J, cudaStream_t s) {
  const size_t tot = (size_t)J * kN * kN;
  const int blocks = (int)std::min<size_t>((tot + kThreads - 1) / kThreads, 4096);
  k_intensity_split<<<blocks, kThreads, 0, s>>>(isplit, inten, J);
  return cudaGetLastError();
}

}  // namespace dmk
