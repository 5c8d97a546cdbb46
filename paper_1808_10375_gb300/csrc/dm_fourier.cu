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
#include "dm_psi.cuh"
#include "dm_ptx.cuh"

namespace dmk {

template <int N>
struct FCfg {
  static constexpr int R1 = FftShape<N>::R1, R2 = FftShape<N>::R2, D = R1 / R2;
  static constexpr int GROUPS = kThreads / R2;          // transforms in flight per CTA
  static constexpr int GR = GROUPS < N ? GROUPS : N;     // rows per row task
  // A row exchange buffer holds the R1 x R2 values of one transform as R1
  // rows of R2 + 1 (one pad element per row): pass 1 of thread t writes
  // row k1 at column t, pass 2 reads column tt of rows t' + R2 d, and both
  // are bank-conflict free with constant offsets from a per-thread base.
  static constexpr int XP = R1 * (R2 + 1);
  // Per-group strides of the exchange buffers and of the plain rows.  A warp
  // holds 32 / R2 groups, each touching R2 consecutive 8-byte values at a
  // time; strides congruent to R2 modulo 16 values (128 bytes, the 32 banks)
  // put the groups of a warp on different banks.  At R2 = 16 one group
  // covers all banks and the strides stay as they are.
  static constexpr int XS = XP + (((R2 - XP) % 16) + 16) % 16;
  static constexpr int NS = N + (((R2 - N) % 16) + 16) % 16;
  static_assert(XS % 2 == 0 && NS % 2 == 0, "row buffers start on 16-byte boundaries");
};

// Row buffers of the row tasks, per group g of R2 lanes: the exchange
// buffer (padded, XP values in a slot of XS), then two plain rows of N
// values (in slots of NS).
template <int N>
__device__ __forceinline__ float2* row_xbuf(float2* stage, int g) { return stage + g * FCfg<N>::XS; }
template <int N>
__device__ __forceinline__ float2* row_buf(float2* stage, int g, int i) {
  using C = FCfg<N>;
  return stage + C::GR * C::XS + (i * C::GR + g) * C::NS;
}

// ------------------------------------------------------------------ R task
// Each group of R2 lanes owns three row buffers: A stages psi of the next
// mode, B stages P of the next mode and doubles as the exchange buffer of the
// transform, O holds the object row (the same for every mode, staged once).
// The copies are asynchronous (psi and P 16-byte, the object row 8-byte as
// it starts at any column); the buffers belong to the group, so only
// warp-level sync is needed.  psi, the stream from DRAM, is requested a whole
// mode ahead; P (L2-resident) once the exchange has freed buffer B.
template <int N, class PsiT = float2>
__device__ __forceinline__ void row_forward(const FourierArgs& a, float2* stage, const float2* twF,
                                            int j, int jj, int rb, float2* slot) {
  using C = FCfg<N>;
  const int g = threadIdx.x / C::R2, t = threadIdx.x % C::R2;
  if (g >= C::GR) return;  // whole idle warps (GR * R2 is a multiple of 32)
  const int y = rb * C::GR + g;
  const int2 p = a.pos[j];
  const float2* orow = a.obj + (size_t)(p.x + y) * a.W + p.y;
  float2* srow_s = row_buf<N>(stage, g, 0);    // A: staged psi row
  float2* prow_s = row_xbuf<N>(stage, g);      // B: staged probe row, then the exchange
  float2* orow_s = row_buf<N>(stage, g, 1);    // O: object row
  float2* xg = prow_s;
  const uint64_t pol_first = l2_policy_evict_first(), pol_last = l2_policy_evict_last();
  // psi rows are N values of PsiT: N * sizeof(PsiT) / 16 copies of 16 bytes
  auto issue_psi = [&](int k) {
    if constexpr (sizeof(PsiT) == sizeof(float2)) {
      const float2* src = static_cast<const float2*>(a.psi) + (((size_t)j * a.M + k) * N + y) * N;
      for (int q = t; q < N / 2; q += C::R2) cp_async16_hint(srow_s + 2 * q, src + 2 * q, pol_first);
    } else {
      constexpr int kPsiChunks = N * (int)sizeof(PsiT) / 16;
      const char* src = reinterpret_cast<const char*>(static_cast<const PsiT*>(a.psi) + (((size_t)j * a.M + k) * N + y) * N);
      char* dst = reinterpret_cast<char*>(srow_s);
      for (int q = t; q < kPsiChunks; q += C::R2) cp_async16_hint(dst + 16 * q, src + 16 * q, pol_first);
    }
  };
  const PsiT* srow_t = reinterpret_cast<const PsiT*>(srow_s);
  auto issue_p = [&](int k) {
    const float2* src = a.probe + ((size_t)k * N + y) * N;
    for (int q = t; q < N / 2; q += C::R2) cp_async16_hint(prow_s + 2 * q, src + 2 * q, pol_last);
  };
  for (int x = t; x < N; x += C::R2) cp_async8(orow_s + x, orow + x);
  issue_psi(0);
  issue_p(0);
  cp_async_commit();
  for (int k = 0; k < a.M; ++k) {
    cp_async_wait<0>();
    __syncwarp();
    float2 v[C::R1];
#pragma unroll
    for (int i = 0; i < C::R1; ++i) {
      const int x = t + C::R2 * i;
      const float2 po = cmul(prow_s[x], orow_s[x]);
      const float2 s = psi_ld(srow_t + x);
      v[i] = make_float2(fmaf(2.f, po.x, -s.x), fmaf(2.f, po.y, -s.y));
    }
    __syncwarp();
    const bool more = k + 1 < a.M;
    if (more) { issue_psi(k + 1); cp_async_commit(); }
    fft_pass1<N, false>(v, t, twF);
#pragma unroll
    for (int k1 = 0; k1 < C::R1; ++k1) xg[k1 * (C::R2 + 1) + t] = v[p1_index<N>(k1)];
    __syncwarp();
#pragma unroll
    for (int d = 0; d < C::D; ++d)
#pragma unroll
      for (int tt = 0; tt < C::R2; ++tt) v[d * C::R2 + tt] = xg[(t + C::R2 * d) * (C::R2 + 1) + tt];
    __syncwarp();
    if (more) { issue_p(k + 1); cp_async_commit(); }
    fft_pass2<N, false>(v);
    float2* trow = slot + (((size_t)jj * a.M + k) * N + y) * N;
#pragma unroll
    for (int d = 0; d < C::D; ++d)
#pragma unroll
      for (int k2 = 0; k2 < C::R2; ++k2) st_cg_hint(trow + t + C::R2 * d + C::R1 * k2, v[p2_index<N>(d, k2)], pol_last);
  }
}

// ------------------------------------------------------------------ I task
// Row buffers as in the R task: A stages U of the next mode and doubles as
// the exchange buffer, B stages P of the next mode, O holds the object row.
// U (L2-resident scratch) is requested once the exchange has freed buffer A;
// P once the current epilogue has used its own.  The object-source sum over
// the modes stays in registers (each thread owns the same positions for every
// mode).  Pending copy groups at the top of mode k: U_k (with the object row
// at k = 0), then P_k.  With PSIERR the old exit waves are read back before
// they are overwritten, and the thread's sums of |psi' - psi|^2 and |psi'|^2
// are returned (zero otherwise).
template <int N, bool PSIERR, class PsiT = float2>
__device__ __forceinline__ float2 row_inverse(const FourierArgs& a, float2* stage, const float2* twF,
                                              int j, int jj, int rb, const float2* slot) {
  using C = FCfg<N>;
  const int g = threadIdx.x / C::R2, t = threadIdx.x % C::R2;
  float2 perr = make_float2(0.f, 0.f);
  if (g >= C::GR) return perr;
  const int y = rb * C::GR + g;
  const int2 p = a.pos[j];
  const float2* orow = a.obj + (size_t)(p.x + y) * a.W + p.y;
  float2* urow_s = row_xbuf<N>(stage, g);      // A: staged row of U, then the exchange
  float2* prow_s = row_buf<N>(stage, g, 0);    // B: staged probe row
  float2* orow_s = row_buf<N>(stage, g, 1);    // O: object row
  float2* xg = urow_s;
  const float c2b = 2.f - a.beta;
  const uint64_t pol_last = l2_policy_evict_last();
  auto stage_row = [&](float2* dst, const float2* src) {
    for (int q = t; q < N / 2; q += C::R2) cp_async16_hint(dst + 2 * q, src + 2 * q, pol_last);
    cp_async_commit();
  };
  auto urow_g = [&](int k) { return slot + (((size_t)jj * a.M + k) * N + y) * N; };
  for (int x = t; x < N; x += C::R2) cp_async8(orow_s + x, orow + x);
  stage_row(urow_s, urow_g(0));
  stage_row(prow_s, a.probe + (size_t)y * N);
  float2 cacc[C::R1];
  for (int k = 0; k < a.M; ++k) {
    cp_async_wait<1>();   // U_k
    __syncwarp();
    // this is the last read of the scratch row: drop its L2 lines unwritten
    for (int q = t; q < N * (int)sizeof(float2) / 128; q += C::R2)
      l2_discard128(reinterpret_cast<const char*>(urow_g(k)) + 128 * q);
    float2 v[C::R1];
#pragma unroll
    for (int i = 0; i < C::R1; ++i) v[i] = urow_s[t + C::R2 * i];
    __syncwarp();
    const bool more = k + 1 < a.M;
    fft_pass1<N, true>(v, t, twF);
#pragma unroll
    for (int k1 = 0; k1 < C::R1; ++k1) xg[k1 * (C::R2 + 1) + t] = v[p1_index<N>(k1)];
    __syncwarp();
#pragma unroll
    for (int d = 0; d < C::D; ++d)
#pragma unroll
      for (int tt = 0; tt < C::R2; ++tt) v[d * C::R2 + tt] = xg[(t + C::R2 * d) * (C::R2 + 1) + tt];
    __syncwarp();
    if (more) stage_row(urow_s, urow_g(k + 1));
    fft_pass2<N, true>(v);
    if (more) cp_async_wait<1>(); else cp_async_wait<0>();   // P_k
    __syncwarp();
    PsiT* srow = static_cast<PsiT*>(a.psi) + (((size_t)j * a.M + k) * N + y) * N;
#pragma unroll
    for (int d = 0; d < C::D; ++d) {
#pragma unroll
      for (int k2 = 0; k2 < C::R2; ++k2) {
        const int x = t + C::R2 * d + C::R1 * k2;
        const float2 pk = prow_s[x];
        const float2 po = cmul(pk, orow_s[x]);
        const float2 g2 = v[p2_index<N>(d, k2)];
        const float2 pn = make_float2(fmaf(c2b, po.x, g2.x), fmaf(c2b, po.y, g2.y));
        if constexpr (PSIERR) {
          const float2 old = psi_ldcs(srow + x);
          const float2 dv = csub(pn, old);
          perr.x += cnorm(dv);
          perr.y += cnorm(pn);
        }
        psi_stcs(srow + x, pn);
        const float2 cn = cconjmul(pk, pn);
        cacc[d * C::R2 + k2] = k == 0 ? cn : cadd(cacc[d * C::R2 + k2], cn);
      }
    }
    __syncwarp();
    if (more) stage_row(prow_s, a.probe + ((size_t)(k + 1) * N + y) * N);
  }
  float2* crow = a.cview + ((size_t)j * N + y) * N;
#pragma unroll
  for (int d = 0; d < C::D; ++d)
#pragma unroll
    for (int k2 = 0; k2 < C::R2; ++k2) __stcs(crow + t + C::R2 * d + C::R1 * k2, cacc[d * C::R2 + k2]);
  return perr;
}

struct Pipe {                     // per-thread bookkeeping of the strip barriers
  uint32_t issued[kMaxStripBufs];  // TMA loads issued on barrier b (one per strip buffer)
  uint32_t done[kMaxStripBufs];    // TMA loads waited for
};

// Wait for the TMA load on barrier b: lane 0 of each warp polls (so that
// spinning warps take few issue slots from co-resident tasks), then every
// lane observes the completed phase itself.  All lanes of the warp call it.
__device__ __forceinline__ void pipe_wait(Pipe& p, uint64_t* bars, int b, int* status) {
  const uint32_t par = p.done[b] & 1u;
  if ((threadIdx.x & 31) == 0) mbar_wait_bounded(&bars[b], par, status);
  __syncwarp();
  (void)mbar_try_wait_parity(&bars[b], par);
  p.done[b]++;
}

// Single-thread form for the drain at the end of the kernel.
__device__ __forceinline__ void pipe_drain(Pipe& p, uint64_t* bars, int b, int* status) {
  mbar_wait_bounded(&bars[b], p.done[b] & 1u, status);
  p.done[b]++;
}

// ------------------------------------------------------------------ C task
// Strips of kStripW = 2 columns of every mode move between the row-major
// scratch and shared memory as 3-D TMA boxes (2 columns x N rows x M modes),
// laid out [mode][row][column]; the task's strips are double- or triple-
// buffered and U goes back with a TMA store.
//
// Each mode of a strip is transformed by 2 R2 threads ("a slot"), lane bit 0
// picking the column, so that every half-warp reads and writes whole 16-byte
// rows of the strip (no bank conflicts in either exchange).  The forward
// column DFT ends in the pass-2 distribution; the modulus projection is
// applied there in registers, and the inverse starts from that distribution
// (ifft_stepA/B), so no reordering exchange sits between the two transforms.
// The mode sum S(q) = sum_k |X_k(q)|^2 is the only cross-slot step: every slot
// writes |X_k|^2, one pass computes the factor (beta s - 1/N^2) per pixel, and
// every slot reads it back.  With more modes than slots (N = 256, M > 8) the
// slots take the modes in rounds and keep X in their part of the strip.
template <int N>
struct CCfg {
  static constexpr int R1 = FftShape<N>::R1, R2 = FftShape<N>::R2, D = R1 / R2;
  static constexpr int TPM = kStripW * R2;     // threads per mode slot
  static constexpr int SLOTS = kThreads / TPM; // modes per round
};

// Strips a column task transforms at once.  With fewer modes than slots G
// strips share the slots, strip q of the gang taking slots q*M .. q*M + M - 1.
// GANG = false compiles the one-strip form (G = 1), which the single-scan
// kernel uses whenever the modes fill the slots by themselves.
template <bool GANG>
__device__ __forceinline__ int col_gang(const FourierArgs& a) { return GANG ? a.G : 1; }
static_assert(kStripW == 2, "the column-task lane layout assumes two columns per strip");

template <int N>
__device__ __forceinline__ unsigned slot_mask() {
  constexpr int TPM = CCfg<N>::TPM;
  if constexpr (TPM >= 32) return 0xffffffffu;
  else return ((1u << TPM) - 1u) << ((threadIdx.x & 31) & ~(TPM - 1));
}

// Forward column DFT of the column this thread's slot lane owns; `base`
// addresses row 0 of that column (row r at base[r * kStripW]).  Returns X in
// the pass-2 distribution.
template <int N>
__device__ __forceinline__ void col_forward(float2* base, int t, const float2* twF, unsigned mask,
                                            float2 (&v)[FftShape<N>::R1]) {
  using C = CCfg<N>;
  constexpr int SW = kStripW;
#pragma unroll
  for (int i = 0; i < C::R1; ++i) v[i] = base[(t + C::R2 * i) * SW];
  fft_pass1<N, false>(v, t, twF);
  __syncwarp(mask);
#pragma unroll
  for (int k1 = 0; k1 < C::R1; ++k1) base[(k1 * C::R2 + (t ^ (k1 & (C::R2 - 1)))) * SW] = v[p1_index<N>(k1)];
  __syncwarp(mask);
#pragma unroll
  for (int d = 0; d < C::D; ++d)
#pragma unroll
    for (int tt = 0; tt < C::R2; ++tt) v[d * C::R2 + tt] = base[((t + C::R2 * d) * C::R2 + (tt ^ t)) * SW];
  fft_pass2<N, false>(v);
}

// Positions a thread owns in its column between the two exchanges (the
// pass-2 read positions): where X waits when the modes take several rounds.
template <int N>
__device__ __forceinline__ int own_row(int t, int r) {
  using C = CCfg<N>;
  const int d = r / C::R2, tt = r % C::R2;
  return (t + C::R2 * d) * C::R2 + (tt ^ t);
}

// Inverse column DFT from the pass-2 distribution; writes x back to the rows
// pass 1 read.
template <int N>
__device__ __forceinline__ void col_inverse(float2* base, int t, const float2* twD, unsigned mask,
                                            float2 (&v)[FftShape<N>::R1]) {
  using C = CCfg<N>;
  constexpr int SW = kStripW;
  ifft_stepA<N>(v, t, twD);
#pragma unroll
  for (int r = 0; r < C::R1; ++r) base[own_row<N>(t, r) * SW] = v[r];
  __syncwarp(mask);
#pragma unroll
  for (int k1 = 0; k1 < C::R1; ++k1) v[k1] = base[(k1 * C::R2 + (t ^ (k1 & (C::R2 - 1)))) * SW];
  __syncwarp(mask);
  ifft_stepB<N>(v);
#pragma unroll
  for (int i = 0; i < C::R1; ++i) base[(t + C::R2 * i) * SW] = v[p1_index<N>(i)];
}

// |X|^2 of this thread's pixels into the mode's norm row (layout [q][column]).
template <int N>
__device__ __forceinline__ void col_norms(float* nrm, int t, int c, const float2 (&v)[FftShape<N>::R1]) {
  using C = CCfg<N>;
#pragma unroll
  for (int d = 0; d < C::D; ++d)
#pragma unroll
    for (int k2 = 0; k2 < C::R2; ++k2) nrm[(t + C::R2 * d + C::R1 * k2) * kStripW + c] = cnorm(v[p2_index<N>(d, k2)]);
}

template <int N>
__device__ __forceinline__ void col_scale(const float* fb, int t, int c, float2 (&v)[FftShape<N>::R1]) {
  using C = CCfg<N>;
#pragma unroll
  for (int d = 0; d < C::D; ++d)
#pragma unroll
    for (int k2 = 0; k2 < C::R2; ++k2) {
      const int q = t + C::R2 * d + C::R1 * k2;
      v[p2_index<N>(d, k2)] = cscale(v[p2_index<N>(d, k2)], fb[q * kStripW + c]);
    }
}

// Modulus factor per pixel p = g * 2N + q * 2 + c of the gang's strips
// (strip g, row q, column c): S = sum_k nrm_{g M + k}[q * 2 + c], the scale
// s = sqrt(I) / (N sqrt(S)) (0 where S = 0) and f = beta s - 1/N^2 into fb[p];
// returns this thread's Fourier-error terms added to `ef`.  MM >= M bounds the
// unrolled mode loop.
template <int N, int MM, bool GANG>
__device__ __forceinline__ float col_factor(const float* nrm, int nstride, const float* ib, float* fb, int M,
                                            int G, float beta, float ef) {
  constexpr int SP = N * kStripW;
  const float invN = 1.f / (float)N;
  const float invN2 = invN * invN;
  for (int p = threadIdx.x; p < G * SP; p += kThreads) {
    const float* ng = GANG ? nrm + (p / SP) * M * nstride + (p % SP) : nrm + p;
    float S = 0.f;
#pragma unroll
    for (int k = 0; k < MM; ++k)
      if (k < M) S += ng[k * nstride];
    // sqrt(I), sqrt(S) and sqrt(I)/sqrt(S) from two reciprocal square roots
    // (rsqrtf, a few ulp): the factor needs FP32 relative accuracy, not
    // correct rounding, and this step sits between two block barriers
    const float iv = ib[p];
    const float ri = rsqrtf(iv), rs = rsqrtf(S);
    const float si_ = iv > 0.f ? iv * ri : 0.f;
    const float ss = S > 0.f ? S * rs : 0.f;
    const float sc = S > 0.f ? si_ * rs * invN : 0.f;
    const float dd = fmaf(ss, invN, -si_);
    ef = fmaf(dd, dd, ef);
    fb[p] = fmaf(beta, sc, -invN2);
  }
  return ef;
}

template <int N, bool GANG>
__device__ __forceinline__ float col_factor_any(const float* nrm, int nstride, const float* ib, float* fb, int M,
                                                int G, float beta, float ef) {
  if (M <= 1) return col_factor<N, 1, GANG>(nrm, nstride, ib, fb, M, G, beta, ef);
  if (M <= 2) return col_factor<N, 2, GANG>(nrm, nstride, ib, fb, M, G, beta, ef);
  if (M <= 4) return col_factor<N, 4, GANG>(nrm, nstride, ib, fb, M, G, beta, ef);
  if (M <= 8) return col_factor<N, 8, GANG>(nrm, nstride, ib, fb, M, G, beta, ef);
  return col_factor<N, kMaxModes, GANG>(nrm, nstride, ib, fb, M, G, beta, ef);
}

// With tmap1 (a box of one mode) and the modes in one round over several
// strip buffers, each slot stores its own mode of U as soon as its inverse is
// done, so no block barrier waits for the slowest mode before the store; a
// slot's leader makes sure its stores have left shared memory before the
// next barrier A (after which the buffer may be refilled), and that they have
// completed before the task ends.  Otherwise thread 0 stores the whole strip
// after barrier C.
template <int N, bool GANG>
__device__ __forceinline__ double column_task(const FourierArgs& a, const CUtensorMap* tmap,
                                              const CUtensorMap* tmap1, float2* sbuf,
                                              float* ibuf, float* fbuf, float* nbuf, const float2* twF,
                                              uint64_t* bars, Pipe& pp, int j, int zview, int sg) {
  using C = CCfg<N>;
  constexpr int SW = kStripW;
  constexpr int SP = N * SW;                  // pixels of one strip
  const int M = a.M;
  const int G = col_gang<GANG>(a);            // strips per buffer (rounds == 1 whenever G > 1)
  const int tid = threadIdx.x;
  const float beta = a.beta;
  const int nbufs = a.strip_bufs;
  const float2* twD = tw_dif<N>(twF);
  const uint32_t strip_elems = (uint32_t)M * N * SW;
  const uint32_t buf_elems = strip_elems * (uint32_t)G;
  const uint32_t strip_bytes = strip_elems * (uint32_t)sizeof(float2);
  const int slot = tid / C::TPM, c = tid & 1, t = (tid >> 1) & (C::R2 - 1);
  const int gq = GANG ? slot / M : 0;         // the slot's strip within the gang
  const unsigned mask = slot_mask<N>();
  const int rounds = (M + C::SLOTS - 1) / C::SLOTS;
  const int nsi = a.SPG / G;                  // gangs of strips in this task
  const bool slot_store = tmap1 != nullptr && rounds == 1 && nbufs > 1;
  const bool leader = (tid & (C::TPM - 1)) == 0 && slot < G * M;   // one lane per busy slot
  // norms: in a single round each slot's part of the strip is free once its
  // forward transform is done; otherwise in the separate buffer
  const int nstride = rounds == 1 ? 2 * N * SW : N * SW;   // floats per mode
  float ef = 0.f;  // this thread's few terms; the cross-thread sums are FP64
  const uint64_t pol_first = l2_policy_evict_first(), pol_last = l2_policy_evict_last();
  auto issue = [&](int si) {  // gang si of the task into buffer si % nbufs (all threads)
    const int s = sg * a.SPG + si * G;
    const int b = si % nbufs;
    if (tid == 0) {
      mbar_arrive_expect_tx(&bars[b], strip_bytes * (uint32_t)G);
      for (int g = 0; g < G; ++g)
        tma_load_3d_hint(sbuf + (size_t)b * buf_elems + (size_t)g * strip_elems, tmap, (s + g) * SW, 0, zview,
                         &bars[b], pol_last);
    }
    pp.issued[b]++;
    const float* ist = a.istrip + ((size_t)j * a.NS + s) * SP;   // the gang's strips are consecutive
    for (int q = tid; q < (G * SP) / 4; q += kThreads)
      cp_async16_hint(ibuf + b * (G * SP) + 4 * q, ist + 4 * q, pol_first);
    cp_async_commit();
  };
  // Every buffer starts with a strip; later strips are issued in the middle
  // of a strip (after barrier A), into the buffer whose TMA store was issued
  // one strip earlier and has long left shared memory, so thread 0 does not
  // wait for a store on the way between strips.
  if (tid == 0) fence_proxy_async_global();
  int issued = 0;
  for (; issued < nbufs && issued < nsi; ++issued) issue(issued);
  for (int si = 0; si < nsi; ++si) {
    const int s = sg * a.SPG + si * G;
    const int b = si % nbufs;
    float2* sb = sbuf + (size_t)b * buf_elems;
    const float* ib = ibuf + b * (G * SP);
    pipe_wait(pp, bars, b, a.status);   // every thread waits for the strip itself
    float* nrm = rounds == 1 ? reinterpret_cast<float*>(sb) : nbuf;
    float2 v[C::R1];
    if (rounds == 1) {
      // slot = g * M + k: strip g of the gang, mode k (laid out in that order)
      if (slot < G * M) {
        float2* base = sb + slot * N * SW + c;
        col_forward<N>(base, t, twF, mask, v);
        __syncwarp(mask);   // the slot's exchange reads are done: its part holds the norms now
        col_norms<N>(nrm + slot * nstride, t, c, v);
      }
    } else {
      for (int r = 0; r < rounds; ++r) {
        const int k = r * C::SLOTS + slot;
        if (k < M) {
          float2* base = sb + k * N * SW + c;
          col_forward<N>(base, t, twF, mask, v);
          col_norms<N>(nrm + k * nstride, t, c, v);
#pragma unroll
          for (int q = 0; q < C::R1; ++q) base[own_row<N>(t, q) * SW] = v[q];
        }
      }
    }
    // intensities of strips after si may still be in flight (one group per strip)
    const int later = issued - si - 1;
    if (later >= 2) cp_async_wait<2>(); else if (later == 1) cp_async_wait<1>(); else cp_async_wait<0>();
    if (slot_store && leader) bulk_wait_read<0>();   // this slot's earlier stores have left the buffers
    __syncthreads();   // A: every mode's norms (and this strip's intensities) are in place
    if (issued < nsi && issued - si < nbufs) {
      // strip `issued` goes to the buffer of strip issued - nbufs <= si - 1,
      // whose store was committed before barrier C of that strip
      if (tid == 0) bulk_wait_read<0>();   // at most the store of strip si - 1 is pending
      issue(issued);
      ++issued;
    }
    ef = col_factor_any<N, GANG>(nrm, nstride, ib, fbuf, M, G, beta, ef);
    __syncthreads();   // B: the factors are in place; the norms are no longer read
    if (rounds == 1) {
      if (slot < G * M) {
        col_scale<N>(fbuf + gq * SP, t, c, v);
        col_inverse<N>(sb + slot * N * SW + c, t, twD, mask, v);
      }
    } else {
      for (int r = 0; r < rounds; ++r) {
        const int k = r * C::SLOTS + slot;
        if (k < M) {
          float2* base = sb + k * N * SW + c;
#pragma unroll
          for (int q = 0; q < C::R1; ++q) v[q] = base[own_row<N>(t, q) * SW];
          col_scale<N>(fbuf, t, c, v);
          col_inverse<N>(base, t, twD, mask, v);
        }
      }
    }
    if (slot_store) {
      // each slot's U goes back on its own once the slot's lanes have written it
      if (slot < G * M) {
        fence_proxy_async_smem();
        __syncwarp(mask);
        if (leader) {
          const int g = GANG ? slot / M : 0, k = GANG ? slot - g * M : slot;
          tma_store_3d_hint(tmap1, (s + g) * SW, 0, zview + k, sb + (size_t)slot * N * SW, pol_last);
          bulk_commit();
        }
      }
      continue;
    }
    fence_proxy_async_smem();
    __syncthreads();   // C: U of every mode is in the strip
    if (tid == 0) {
      for (int g = 0; g < G; ++g) tma_store_3d_hint(tmap, (s + g) * SW, 0, zview, sb + (size_t)g * strip_elems, pol_last);
      bulk_commit();
    }
    if (nbufs == 1 && issued < nsi) {
      // a single buffer: the next strip waits for this store to leave it
      if (tid == 0) bulk_wait_read<0>();
      issue(issued);
      ++issued;
    }
  }
  if (slot_store && leader) bulk_wait<0>();   // the slot's stores are complete before the task is published
  return (double)ef;
}

// The persistent task loop over several scans of frame size N.  Scan s
// owns tasks [base[s], base[s+1]) of the launch's counter `disp`; within a
// scan the order and dependencies are those of its own plan (stage offsets,
// per-chunk counters, scratch ring).  A CTA's tasks increase, so it moves
// through the scans in order.
template <int N>
__device__ __forceinline__ void fourier_tasks(const FourierArgs* as, const CUtensorMap* maps, const int* base,
                                              int nscan, int* disp) {
  extern __shared__ unsigned char smem_raw[];
  // 128-byte aligned base (TMA boxes land at 128-byte aligned addresses)
  float2* tw = reinterpret_cast<float2*>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
  float2* work = tw + kTwBytes / sizeof(float2);
  // row tasks: three row buffers per transform; column tasks: the strip
  // buffers, then their intensities, the modulus factors and (with several
  // rounds of modes) the norms, laid out for the scan of the task
  float2* stage = work;
  float2* sbuf = work;
  __shared__ __align__(8) uint64_t bars[kMaxStripBufs];
  __shared__ int s_task;
  __shared__ int s_skip;
  __shared__ double s_red[kThreads / 32];
  for (int i = threadIdx.x; i < tw_entries<N>(); i += kThreads) tw[i] = as[0].tw[i];
  if (threadIdx.x == 0) {
    for (int b = 0; b < kMaxStripBufs; ++b) mbar_init(&bars[b], 1);
    fence_mbar_init();
  }
  Pipe pp = {};
  const int total = base[nscan];
  int next = 0;
  if (threadIdx.x == 0) next = atomicAdd(disp, 1);
  int st_prev = 0, scan_prev = 0;

  for (;;) {
    if (threadIdx.x == 0) {
      s_task = next;
      if (next < total) next = atomicAdd(disp, 1);
    }
    __syncthreads();
    const int gtask = s_task;
    if (gtask >= total) break;
    int sc = scan_prev;
    while (base[sc + 1] <= gtask) ++sc;
    if (sc != scan_prev) { scan_prev = sc; st_prev = 0; }
    const FourierArgs& a = as[sc];
    const int task = gtask - base[sc];
    int* doneR = a.counters + 1;   // completion counters per view
    int* doneC = doneR + a.J;
    int* doneI = doneC + a.J;
    const size_t slot_elems = (size_t)a.B * a.M * N * N;

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
    const int jv = c * a.B + local / (kind == 1 ? a.CG : a.RB);   // the task's view

    // Wait for what this task consumes (the producers of its own view).
    if (threadIdx.x == 0) {
      bool ok = true;
      if (kind == 0) {
        if (c >= a.nslot) ok = spin_wait_geq(doneI + (jv - a.nslot * a.B), a.RB, a.status);
      } else if (kind == 1) {
        ok = spin_wait_geq(doneR + jv, a.RB, a.status);
      } else {
        ok = spin_wait_geq(doneC + jv, a.CG, a.status);
      }
      s_skip = ok ? 0 : 1;
    }
    __syncthreads();

    if (!s_skip) {
      const int sl = c % a.nslot;
      float2* slot = a.scratch + (size_t)sl * slot_elems;
      if (kind == 0) {
        const int jj = local / a.RB, rb = local % a.RB;
        row_forward<N>(a, stage, tw, c * a.B + jj, jj, rb, slot);
      } else if (kind == 1) {
        const int jj = local / a.CG, sg = local % a.CG;
        const int j = c * a.B + jj;
        const int G = col_gang<true>(a);
        float* ibuf = reinterpret_cast<float*>(work + (size_t)a.strip_bufs * G * a.M * N * kStripW);
        float* fbuf = ibuf + (size_t)a.strip_bufs * G * N * kStripW;   // modulus factors of the current gang
        float* nbuf = fbuf + N * kStripW;                              // norms when the modes take several rounds
        double ef = column_task<N, true>(a, maps + sc, nullptr, sbuf, ibuf, fbuf, nbuf, tw, bars, pp, j,
                                         (sl * a.B + jj) * a.M, sg);
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
        row_inverse<N, false>(a, stage, tw, c * a.B + jj, jj, rb, slot);
      }
    }
    // Publish the task: the barrier orders every thread's writes before
    // thread 0's device-scope fence and counter update (a release by one
    // thread after the barrier covers the whole CTA).
    __syncthreads();
    if (threadIdx.x == 0) {
      bulk_wait<0>();   // TMA stores of the task have landed
      __threadfence();
      atomicAdd((kind == 0 ? doneR : kind == 1 ? doneC : doneI) + jv, 1);
    }
  }
  // Copies that a timed-out wait left in flight must land before the CTA exits.
  if (threadIdx.x == 0) {
    for (int b = 0; b < kMaxStripBufs; ++b)
      while (pp.done[b] < pp.issued[b]) pipe_drain(pp, bars, b, as[0].status);
    bulk_wait<0>();
  }
}

// One scan: the same task loop as fourier_tasks, specialised to one scan
// whose arguments are the kernel's own parameters (which keeps its register
// allocation lean); its task counter is counters[0].
template <int N, bool GANG, bool PSIERR, class PsiT = float2>
__global__ void __launch_bounds__(kThreads, 2)
    k_fourier(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap tmap1,
              const FourierArgs a) {
  using C = FCfg<N>;
  extern __shared__ unsigned char smem_raw[];
  // 128-byte aligned base (TMA boxes land at 128-byte aligned addresses)
  float2* tw = reinterpret_cast<float2*>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
  float2* work = tw + kTwBytes / sizeof(float2);
  // row tasks: exchange buffers, then two row buffers per transform (staged
  // psi and P rows of R; the object-source accumulator of I); column tasks:
  // the strip buffers, then their intensities
  float2* stage = work;
  float2* sbuf = work;
  const int G = col_gang<GANG>(a);
  float* ibuf = reinterpret_cast<float*>(work + (size_t)a.strip_bufs * G * a.M * N * kStripW);
  float* fbuf = ibuf + (size_t)a.strip_bufs * G * N * kStripW;   // modulus factors of the current gang
  float* nbuf = fbuf + N * kStripW;                              // norms when the modes take several rounds
  __shared__ __align__(8) uint64_t bars[kMaxStripBufs];
  __shared__ int s_task;
  __shared__ int s_skip;
  __shared__ double s_red[kThreads / 32];
  for (int i = threadIdx.x; i < tw_entries<N>(); i += kThreads) tw[i] = a.tw[i];
  if (threadIdx.x == 0) {
    for (int b = 0; b < kMaxStripBufs; ++b) mbar_init(&bars[b], 1);
    fence_mbar_init();
  }
  Pipe pp = {};

  // per-view completion counters: a column task waits for the row tasks of
  // its own view only (and so on), not for the slowest task of its chunk
  int* disp = a.counters;
  int* doneR = a.counters + 1;
  int* doneC = doneR + a.J;
  int* doneI = doneC + a.J;
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
    const int jv = c * a.B + local / (kind == 1 ? a.CG : a.RB);   // the task's view

    // Wait for what this task consumes.
    if (threadIdx.x == 0) {
      bool ok = true;
      if (kind == 0) {
        // the slot's area of this view was last used by view jv - nslot B
        if (c >= a.nslot) ok = spin_wait_geq(doneI + (jv - a.nslot * a.B), a.RB, a.status);
      } else if (kind == 1) {
        ok = spin_wait_geq(doneR + jv, a.RB, a.status);
      } else {
        ok = spin_wait_geq(doneC + jv, a.CG, a.status);
      }
      s_skip = ok ? 0 : 1;
    }
    __syncthreads();

    if (!s_skip) {
      const int sl = c % a.nslot;
      float2* slot = a.scratch + (size_t)sl * slot_elems;
      if (kind == 0) {
        const int jj = local / a.RB, rb = local % a.RB;
        row_forward<N, PsiT>(a, stage, tw, c * a.B + jj, jj, rb, slot);
      } else if (kind == 1) {
        const int jj = local / a.CG, sg = local % a.CG;
        const int j = c * a.B + jj;
        double ef = column_task<N, GANG>(a, &tmap, &tmap1, sbuf, ibuf, fbuf, nbuf, tw, bars, pp, j,
                                         (sl * a.B + jj) * a.M, sg);
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
        const float2 pe = row_inverse<N, PSIERR, PsiT>(a, stage, tw, c * a.B + jj, jj, rb, slot);
        if constexpr (PSIERR) {
          // this task's exit-wave change sums, in FP64 across the CTA
          double d2 = pe.x, n2 = pe.y;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            d2 += __shfl_xor_sync(0xffffffffu, d2, o);
            n2 += __shfl_xor_sync(0xffffffffu, n2, o);
          }
          __shared__ double s_pe[2][kThreads / 32];
          if ((threadIdx.x & 31) == 0) { s_pe[0][threadIdx.x >> 5] = d2; s_pe[1][threadIdx.x >> 5] = n2; }
          __syncthreads();
          if (threadIdx.x == 0) {
            double td = 0.0, tn = 0.0;
            for (int i = 0; i < kThreads / 32; ++i) { td += s_pe[0][i]; tn += s_pe[1][i]; }
            double* out = a.psi_part + 2 * ((size_t)(c * a.B + jj) * a.RB + rb);
            out[0] = td;
            out[1] = tn;
          }
        }
      }
    }
    // Publish the task: the barrier orders every thread's writes before
    // thread 0's device-scope fence and counter update (a release by one
    // thread after the barrier covers the whole CTA).
    __syncthreads();
    if (threadIdx.x == 0) {
      bulk_wait<0>();   // TMA stores of the task have landed
      __threadfence();
      atomicAdd((kind == 0 ? doneR : kind == 1 ? doneC : doneI) + jv, 1);
    }
  }
  // Copies that a timed-out wait left in flight must land before the CTA exits.
  if (threadIdx.x == 0) {
    for (int b = 0; b < kMaxStripBufs; ++b)
      while (pp.done[b] < pp.issued[b]) pipe_drain(pp, bars, b, a.status);
    bulk_wait<0>();
  }
}

// Several scans of the same frame size in one persistent launch.
template <int N>
__global__ void __launch_bounds__(kThreads, 2) k_fourier_batch(const __grid_constant__ FourierBatch b) {
  fourier_tasks<N>(b.a, b.map, b.base, b.nscan, b.dispenser);
}

template <int N>
static int tw_host(float2* tab) {
  if (tab)
    tw_fill<N>(tab, [](int m) {
      const double ang = -2.0 * 3.14159265358979323846 * (double)m / (double)N;
      return make_float2((float)cos(ang), (float)sin(ang));
    });
  return tw_entries<N>();
}

int fourier_twiddles(int N, float2* tab) {
  switch (N) {
    case 16: return tw_host<16>(tab);
    case 32: return tw_host<32>(tab);
    case 64: return tw_host<64>(tab);
    case 128: return tw_host<128>(tab);
    case 256: return tw_host<256>(tab);
    default: return 0;
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
static size_t smem_for(int M, int bufs, int G) {
  using C = FCfg<N>;
  static_assert(tw_entries<N>() * sizeof(float2) <= kTwBytes, "twiddle tables exceed their shared area");
  const size_t rows = sizeof(float2) * (size_t)C::GR * (C::XS + 2 * C::NS);   // three row buffers per transform
  const bool multi = M > CCfg<N>::SLOTS;
  const size_t cols = sizeof(float2) * (size_t)bufs * G * M * N * kStripW  // strips
                      + sizeof(float) * (size_t)bufs * G * N * kStripW     // their intensities
                      + sizeof(float) * (size_t)G * N * kStripW            // modulus factors
                      + (multi ? sizeof(float) * (size_t)M * N * kStripW : 0);  // norms (several rounds)
  return 128 + kTwBytes + (rows > cols ? rows : cols);
}

size_t fourier_smem_bytes(int N, int M, int bufs, int G) {
  switch (N) {
    case 16: return smem_for<16>(M, bufs, G);
    case 32: return smem_for<32>(M, bufs, G);
    case 64: return smem_for<64>(M, bufs, G);
    case 128: return smem_for<128>(M, bufs, G);
    case 256: return smem_for<256>(M, bufs, G);
    default: return 0;
  }
}

// The single-scan kernel: the gang form for every frame size, and for
// N = 256 also the one-strip form (the modes fill the slots by themselves);
// each with and without the exit-wave change sums.  The mixed-precision
// form (exit waves stored as complex half) exists for N = 64, 128 and 256,
// without the exit-wave change sums.
template <bool PSIERR>
static const void* fourier_kernel_t(int N, bool gang) {
  switch (N) {
    case 16: return (const void*)k_fourier<16, true, PSIERR>;
    case 32: return (const void*)k_fourier<32, true, PSIERR>;
    case 64: return (const void*)k_fourier<64, true, PSIERR>;
    case 128: return (const void*)k_fourier<128, true, PSIERR>;
    case 256: return gang ? (const void*)k_fourier<256, true, PSIERR> : (const void*)k_fourier<256, false, PSIERR>;
    default: return nullptr;
  }
}

static const void* fourier_kernel_h(int N, bool gang) {
  switch (N) {
    case 64: return (const void*)k_fourier<64, true, false, __half2>;
    case 128: return (const void*)k_fourier<128, true, false, __half2>;
    case 256: return gang ? (const void*)k_fourier<256, true, false, __half2>
                          : (const void*)k_fourier<256, false, false, __half2>;
    default: return nullptr;
  }
}

bool fourier_has_psi16(int N) { return N == 64 || N == 128 || N == 256; }

static const void* fourier_kernel(int N, bool gang, bool psierr, bool psi16) {
  if (psi16) return psierr ? nullptr : fourier_kernel_h(N, gang);
  return psierr ? fourier_kernel_t<true>(N, gang) : fourier_kernel_t<false>(N, gang);
}

// The dynamic shared-memory limit is a property of the kernel, shared by
// every context that launches it: set it to the device's opt-in maximum so
// that plans of different sizes can all launch.
static cudaError_t allow_max_smem(const void* f) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - 1024);
  return e;
}

// Resident CTAs per SM of the single-scan kernel (the smallest over its
// forms), with every form's shared-memory limit set.
int fourier_occupancy(int N, size_t smem) {
  int best = -1;
  for (int form = 0; form < 3; ++form)   // FP32, FP32 with the exit-wave change, complex-half exit waves
    for (bool gang : {true, false}) {
      if (form == 2 && !fourier_has_psi16(N)) continue;
      const void* f = fourier_kernel(N, gang, form == 1, form == 2);
      if (!f) return 0;
      if (allow_max_smem(f) != cudaSuccess) return 0;
      int nb = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, kThreads, smem) != cudaSuccess) return 0;
      best = best < 0 ? nb : (nb < best ? nb : best);
    }
  return best;
}

static const void* fourier_batch_kernel(int N) {
  switch (N) {
    case 16: return (const void*)k_fourier_batch<16>;
    case 32: return (const void*)k_fourier_batch<32>;
    case 64: return (const void*)k_fourier_batch<64>;
    case 128: return (const void*)k_fourier_batch<128>;
    case 256: return (const void*)k_fourier_batch<256>;
    default: return nullptr;
  }
}

cudaError_t launch_fourier_batch(const FourierBatch& b, int N, int grid, size_t smem, cudaStream_t s) {
  const void* f = fourier_batch_kernel(N);
  if (!f) return cudaErrorInvalidValue;
  cudaError_t e = allow_max_smem(f);
  if (e != cudaSuccess) return e;
  switch (N) {
    case 16: k_fourier_batch<16><<<grid, kThreads, smem, s>>>(b); break;
    case 32: k_fourier_batch<32><<<grid, kThreads, smem, s>>>(b); break;
    case 64: k_fourier_batch<64><<<grid, kThreads, smem, s>>>(b); break;
    case 128: k_fourier_batch<128><<<grid, kThreads, smem, s>>>(b); break;
    case 256: k_fourier_batch<256><<<grid, kThreads, smem, s>>>(b); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

int fourier_batch_occupancy(int N, size_t smem) {
  const void* f = fourier_batch_kernel(N);
  if (!f) return 0;
  if (allow_max_smem(f) != cudaSuccess) return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, kThreads, smem) != cudaSuccess) return 0;
  return nb;
}

template <bool PSIERR>
static cudaError_t launch_fourier_t(const CUtensorMap& m, const CUtensorMap& m1, const FourierArgs& a, int grid,
                                    size_t smem, cudaStream_t s) {
  switch (a.N) {
    case 16: k_fourier<16, true, PSIERR><<<grid, kThreads, smem, s>>>(m, m1, a); break;
    case 32: k_fourier<32, true, PSIERR><<<grid, kThreads, smem, s>>>(m, m1, a); break;
    case 64: k_fourier<64, true, PSIERR><<<grid, kThreads, smem, s>>>(m, m1, a); break;
    case 128: k_fourier<128, true, PSIERR><<<grid, kThreads, smem, s>>>(m, m1, a); break;
    case 256:
      if (a.G > 1) k_fourier<256, true, PSIERR><<<grid, kThreads, smem, s>>>(m, m1, a);
      else k_fourier<256, false, PSIERR><<<grid, kThreads, smem, s>>>(m, m1, a);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

static cudaError_t launch_fourier_h(const CUtensorMap& m, const CUtensorMap& m1, const FourierArgs& a, int grid,
                                    size_t smem, cudaStream_t s) {
  switch (a.N) {
    case 64: k_fourier<64, true, false, __half2><<<grid, kThreads, smem, s>>>(m, m1, a); break;
    case 128: k_fourier<128, true, false, __half2><<<grid, kThreads, smem, s>>>(m, m1, a); break;
    case 256:
      if (a.G > 1) k_fourier<256, true, false, __half2><<<grid, kThreads, smem, s>>>(m, m1, a);
      else k_fourier<256, false, false, __half2><<<grid, kThreads, smem, s>>>(m, m1, a);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// The instance follows the plan: the gang form when G > 1, the exit-wave
// change sums when a.psi_part is set, complex-half exit waves when a.psi16.
cudaError_t launch_fourier(const void* tmaps, const FourierArgs& a, int grid, size_t smem, cudaStream_t s) {
  const CUtensorMap* m = static_cast<const CUtensorMap*>(tmaps);
  if (a.psi16) return a.psi_part ? cudaErrorInvalidValue : launch_fourier_h(m[0], m[1], a, grid, smem, s);
  return a.psi_part ? launch_fourier_t<true>(m[0], m[1], a, grid, smem, s)
                    : launch_fourier_t<false>(m[0], m[1], a, grid, smem, s);
}

}  // namespace dmk
