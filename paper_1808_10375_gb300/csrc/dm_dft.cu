// Batched 2-D DFT of 256 x 256 complex frames, in two precision forms: the
// FP32 register radix-16 FFT of the Fourier step, and a split-precision
// tensor-core form (the reduced-precision DFT the paper's future-work note on
// single precision leads to, Sec. V).
//
// Both run as two passes of one kernel that transforms the 256-point rows of
// a 16-row tile and stores the tile transposed: applied twice (input -> work
// -> output) this is the 2-D transform in the input's orientation.
//
// A 256-point transform is two radix-16 stages (n = t + 16 n2,
// X[k1 + 16 k2] = sum_t W16^(t k2) W256^(t k1) sum_n2 x[t + 16 n2] W16^(n2 k1)).
// In the tensor-core form each stage is the complex product of the 16 x 16
// DFT matrix F with a 16 x L block of data (L lines), computed as real GEMMs
//   Re Y = Fr Xr - Fi Xi,  Im Y = Fi Xr + Fr Xi
// on mma.sync m16n8k16 with BF16 operands and FP32 accumulation.  Every
// operand is split a = a_hi + a_lo (a_hi = bf16(a), a_lo = bf16(a - a_hi)) and
// each real product takes the three terms hi*hi + hi*lo + lo*hi.  The
// W256 twiddles between the stages are applied in FP32 on the CUDA cores.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "dm.h"
#include "dm_fft.cuh"
#include "dm_kernels.h"
#include "dm_ptx.cuh"

namespace dmk {

constexpr int kDftN = 256;
constexpr int kDftRows = 16;     // rows per CTA tile
constexpr int kTileElems = kDftRows * kDftN;
constexpr int kZsPad = kDftRows + 1;   // FP32 form's output tile row (float2): conflict-free transposed writes
constexpr size_t kDftSmem = (size_t)(kTileElems + kDftN * kZsPad) * sizeof(float2);   // exchange tile + output tile

// W256^m (m < 256) and the pass-1 table of the register FFT (twF, [k1][t]),
// filled once per device from double-precision angles.
__device__ float2 g_dft_w[kDftN];
__device__ float2 g_dft_twf[kDftN];

// bf16 x2 register from two floats (low half = first)
__device__ __forceinline__ uint32_t pack_bf16(float lo_part, float hi_part) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo_part, hi_part);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// Split a pair of floats into bf16 x2 (hi) and bf16 x2 (lo) registers.
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat16 ah = __float2bfloat16_rn(a), bh = __float2bfloat16_rn(b);
  __nv_bfloat162 h;
  h.x = ah;
  h.y = bh;
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = pack_bf16(a - __bfloat162float(ah), b - __bfloat162float(bh));
}

// D += A * B with A 16x16 (row-major fragments a[4]), B 16x8 (b[2]), D 16x8 FP32.
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// A fragments of the 16-point DFT matrix F[m][k] = exp(-+2 pi i m k / 16):
// real part hi/lo, imaginary part hi/lo and the negated imaginary part hi/lo.
// Lane (g = lane/4, q = lane%4) holds rows g, g+8 and columns 2q, 2q+1,
// 2q+8, 2q+9 (the m16n8k16 A layout).
struct DftFrags {
  uint32_t rh[4], rl[4], ih[4], il[4], nih[4], nil[4];
};

template <bool INV>
__device__ __forceinline__ void dft_frags(DftFrags& f, int lane) {
  const int g = lane >> 2, q = lane & 3;
  const int rows[2] = {g, g + 8};
  const int cols[2] = {2 * q, 2 * q + 8};
  for (int ri = 0; ri < 2; ++ri)
    for (int ci = 0; ci < 2; ++ci) {
      const int idx = ci * 2 + ri;   // a0a1: (g, 2q..), a2a3: (g+8, 2q..), a4a5: (g, 2q+8..), a6a7: (g+8, 2q+8..)
      float re[2], im[2];
      for (int e = 0; e < 2; ++e) {
        const int m = rows[ri], k = cols[ci] + e;
        double s, c;
        sincospi((double)((m * k) % 16) / 8.0, &s, &c);   // angle 2 pi m k / 16
        re[e] = (float)c;
        im[e] = INV ? (float)s : -(float)s;
      }
      split2(re[0], re[1], f.rh[idx], f.rl[idx]);
      split2(im[0], im[1], f.ih[idx], f.il[idx]);
      split2(-im[0], -im[1], f.nih[idx], f.nil[idx]);
    }
}

// The split fragments of F for both directions, per lane, built once per
// device (FP64 angles are slow on this GPU: built in every CTA they cost
// more than the transform): g_dft_frag[inv][part][register][lane], parts in
// DftFrags order.
__device__ uint32_t g_dft_frag[2][6][4][32];

__global__ void k_dft_tables() {
  const int m = threadIdx.x;   // 256 threads
  double s, c;
  sincospi(-2.0 * (double)m / kDftN, &s, &c);
  g_dft_w[m] = make_float2((float)c, (float)s);
  const int k1 = m / 16, t = m % 16;
  sincospi(-2.0 * (double)((t * k1) % kDftN) / kDftN, &s, &c);
  g_dft_twf[m] = make_float2((float)c, (float)s);
  if (m < 64) {
    const int lane = m & 31, inv = m >> 5;
    DftFrags f;
    if (inv) dft_frags<true>(f, lane); else dft_frags<false>(f, lane);
    for (int i = 0; i < 4; ++i) {
      g_dft_frag[inv][0][i][lane] = f.rh[i];
      g_dft_frag[inv][1][i][lane] = f.rl[i];
      g_dft_frag[inv][2][i][lane] = f.ih[i];
      g_dft_frag[inv][3][i][lane] = f.il[i];
      g_dft_frag[inv][4][i][lane] = f.nih[i];
      g_dft_frag[inv][5][i][lane] = f.nil[i];
    }
  }
}

template <bool INV>
__device__ __forceinline__ void load_frags(DftFrags& f, int lane) {
  const int d = INV ? 1 : 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    f.rh[i] = g_dft_frag[d][0][i][lane];
    f.rl[i] = g_dft_frag[d][1][i][lane];
    f.ih[i] = g_dft_frag[d][2][i][lane];
    f.il[i] = g_dft_frag[d][3][i][lane];
    f.nih[i] = g_dft_frag[d][4][i][lane];
    f.nil[i] = g_dft_frag[d][5][i][lane];
  }
}

// One complex 16-point DFT of 8 lines: B fragments (real/imag, hi/lo) in,
// FP32 accumulators (real/imag) out, 12 tensor-core products.
__device__ __forceinline__ void dft16_tc(const DftFrags& f, const uint32_t (&xr)[2][2], const uint32_t (&xi)[2][2],
                                         float (&yr)[4], float (&yi)[4]) {
  // xr[hl][j]: hl = 0 hi, 1 lo; j = B register 0 (k = 2q, 2q+1) or 1 (k = 2q+8, 2q+9)
  for (int e = 0; e < 4; ++e) { yr[e] = 0.f; yi[e] = 0.f; }
  mma_bf16(yr, f.rh, xr[0][0], xr[0][1]);
  mma_bf16(yr, f.rh, xr[1][0], xr[1][1]);
  mma_bf16(yr, f.rl, xr[0][0], xr[0][1]);
  mma_bf16(yr, f.nih, xi[0][0], xi[0][1]);
  mma_bf16(yr, f.nih, xi[1][0], xi[1][1]);
  mma_bf16(yr, f.nil, xi[0][0], xi[0][1]);
  mma_bf16(yi, f.ih, xr[0][0], xr[0][1]);
  mma_bf16(yi, f.ih, xr[1][0], xr[1][1]);
  mma_bf16(yi, f.il, xr[0][0], xr[0][1]);
  mma_bf16(yi, f.rh, xi[0][0], xi[0][1]);
  mma_bf16(yi, f.rh, xi[1][0], xi[1][1]);
  mma_bf16(yi, f.rl, xi[0][0], xi[0][1]);
}

// Operand planes of the tensor form.  Both stages multiply F by 256 lines of
// 16 values each (stage A: line (r, t) holds x[r][t + 16 n2] over n2; stage
// B: line (r, k1) holds the twiddled stage-A output over t).  The values are
// split once, when a stage's input is written, into four BF16 planes (real
// hi, real lo, imaginary hi, imaginary lo); a line is 32 bytes of a plane
// (two 16-byte chunks: k = 0..7 and k = 8..15), and chunk c of line L sits at
// chunk 2 L + (c ^ ((L >> 2) & 1)), so that the eight lines one ldmatrix
// phase reads cover all 32 banks.  ldmatrix then hands each lane its B
// fragments directly (lane g*4 + q: line g, k = 2q, 2q+1 and 2q+8, 2q+9).
constexpr int kPlaneWords = 256 * 8;              // 32-bit words of one plane (256 lines x 32 bytes)
constexpr int kZsRow = 321;                       // output tile row stride (float2), odd: conflict-free reads
constexpr int kZsK2 = 20;                         // output tile stride of k2 (float2)
constexpr size_t kDftTcSmem = 128 + (size_t)kTileElems * sizeof(float2) + 4 * kPlaneWords * sizeof(uint32_t) +
                              (size_t)kDftRows * kZsRow * sizeof(float2);

__device__ __forceinline__ int plane_word(int line, int w) {   // w: word (two k values), 0..7
  return line * 8 + ((((w >> 2) ^ (line >> 2)) & 1) << 2) + (w & 3);
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

// B fragments (hi and lo, real and imaginary) of lines L0 .. L0 + 7: two
// ldmatrix.x4, each lane supplying one row address (lane = 8 * matrix + row;
// matrices: hi chunk 0, hi chunk 1, lo chunk 0, lo chunk 1).
__device__ __forceinline__ void load_b_planes(const uint32_t* planes, int L0, int lane, uint32_t (&xr)[2][2],
                                              uint32_t (&xi)[2][2]) {
  const int mi = lane >> 3, line = L0 + (lane & 7);
  const int word = plane_word(line, (mi & 1) * 4);
  const uint32_t re = smem_u32(planes + (mi >> 1) * kPlaneWords + word);
  const uint32_t im = smem_u32(planes + (2 + (mi >> 1)) * kPlaneWords + word);
  ldsm_x4(re, xr[0][0], xr[0][1], xr[1][0], xr[1][1]);
  ldsm_x4(im, xi[0][0], xi[0][1], xi[1][0], xi[1][1]);
}

// Two consecutive values of a line (k, k + 1) into the four planes.
__device__ __forceinline__ void store_planes(uint32_t* planes, int line, int w, float2 a, float2 b) {
  uint32_t rh, rl, ih, il;
  split2(a.x, b.x, rh, rl);
  split2(a.y, b.y, ih, il);
  const int o = plane_word(line, w);
  planes[o] = rh;
  planes[kPlaneWords + o] = rl;
  planes[2 * kPlaneWords + o] = ih;
  planes[3 * kPlaneWords + o] = il;
}

// Tensor-core row pass: 16 rows of frame `f` of `in` -> the same 16 columns of
// frame f of `out` (out[f][k][r0 + r] = DFT(in[f][r0 + r])[k]).
template <bool INV>
__global__ void __launch_bounds__(kThreads, 2) k_dft256_rows_tc(const float2* __restrict__ in,
                                                                 float2* __restrict__ out) {
  extern __shared__ unsigned char dft_raw[];
  float2* xs = reinterpret_cast<float2*>(dft_raw + ((128u - (smem_u32(dft_raw) & 127u)) & 127u));   // input tile [r][x]
  uint32_t* planes = reinterpret_cast<uint32_t*>(xs + kTileElems);                                 // 4 operand planes
  float2* zs = reinterpret_cast<float2*>(planes + 4 * kPlaneWords);                                 // output [r][k2 * 20 + k1]
  const float2* tw256 = g_dft_w;
  const int f = blockIdx.x / (kDftN / kDftRows), r0 = (blockIdx.x % (kDftN / kDftRows)) * kDftRows;
  const float2* src = in + ((size_t)f * kDftN + r0) * kDftN;
  for (int i = threadIdx.x; i < kTileElems; i += kThreads) xs[i] = src[i];
  DftFrags fr;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  load_frags<INV>(fr, lane);
  __syncthreads();
  // stage-A planes: line r * 16 + t, k = n2 (pairs n2 = 2w, 2w + 1)
  for (int p = threadIdx.x; p < kTileElems / 2; p += kThreads) {
    const int t = p & 15, w = (p >> 4) & 7, r = p >> 7;
    const float2* row = xs + r * kDftN + t;
    store_planes(planes, r * 16 + t, w, row[16 * (2 * w)], row[16 * (2 * w + 1)]);
  }
  __syncthreads();
  const int g = lane >> 2, q = lane & 3;
  // stage A: lines (r, t), 32 groups of 8 (fixed r, t = t0 .. t0 + 7)
  float ya_r[4][4], ya_i[4][4];
#pragma unroll
  for (int gi = 0; gi < 4; ++gi) {
    const int lg = warp * 4 + gi, r = lg >> 1, t0 = (lg & 1) * 8;
    uint32_t xr[2][2], xi[2][2];
    load_b_planes(planes, r * 16 + t0, lane, xr, xi);
    dft16_tc(fr, xr, xi, ya_r[gi], ya_i[gi]);
  }
  __syncthreads();   // every stage-A operand is read: the planes take the stage-B operands
#pragma unroll
  for (int gi = 0; gi < 4; ++gi) {
    const int lg = warp * 4 + gi, r = lg >> 1, t0 = (lg & 1) * 8;
    // accumulator e: row k1 = g (e < 2) or g + 8, line t = t0 + 2q + (e & 1)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k1 = g + 8 * h, ta = t0 + 2 * q;
      const float2 ya = ctw<INV>(make_float2(ya_r[gi][2 * h], ya_i[gi][2 * h]), tw256[(ta * k1) & 255]);
      const float2 yb = ctw<INV>(make_float2(ya_r[gi][2 * h + 1], ya_i[gi][2 * h + 1]), tw256[((ta + 1) * k1) & 255]);
      // stage-B line r * 16 + k1, k = t (word t / 2)
      store_planes(planes, r * 16 + k1, ta >> 1, ya, yb);
    }
  }
  __syncthreads();
  // stage B: lines (r, k1), 32 groups of 8 (fixed r, k1 = k10 .. k10 + 7)
#pragma unroll
  for (int gi = 0; gi < 4; ++gi) {
    const int lg = warp * 4 + gi, r = lg >> 1, k10 = (lg & 1) * 8;
    uint32_t xr[2][2], xi[2][2];
    load_b_planes(planes, r * 16 + k10, lane, xr, xi);
    float yr[4], yi[4];
    dft16_tc(fr, xr, xi, yr, yi);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int k2 = g + ((e >> 1) << 3), k1 = k10 + 2 * q + (e & 1);
      zs[r * kZsRow + k2 * kZsK2 + k1] = make_float2(yr[e], yi[e]);
    }
  }
  __syncthreads();
  float2* dst = out + (size_t)f * kDftN * kDftN + r0;
  for (int i = threadIdx.x; i < kTileElems; i += kThreads) {
    const int k = i / kDftRows, r = i % kDftRows;
    dst[(size_t)k * kDftN + r] = zs[r * kZsRow + (k >> 4) * kZsK2 + (k & 15)];
  }
}

// FP32 row pass with the register radix-16 FFT of the Fourier step.
template <bool INV>
__global__ void __launch_bounds__(kThreads) k_dft256_rows_fp32(const float2* __restrict__ in,
                                                                float2* __restrict__ out) {
  constexpr int R1 = FftShape<kDftN>::R1, R2 = FftShape<kDftN>::R2;
  extern __shared__ float2 dft_smem[];
  float2* xs = dft_smem;                // exchange buffers [row][N]
  float2* zs = dft_smem + kTileElems;   // output tile [k][r], rows of kZsPad
  __shared__ float2 tw[kDftN];
  const int f = blockIdx.x / (kDftN / kDftRows), r0 = (blockIdx.x % (kDftN / kDftRows)) * kDftRows;
  for (int i = threadIdx.x; i < kDftN; i += kThreads) tw[i] = g_dft_twf[i];
  __syncthreads();
  const int gr = threadIdx.x / R2, t = threadIdx.x % R2;   // row of the tile, lane in the transform
  const float2* src = in + ((size_t)f * kDftN + r0 + gr) * kDftN;
  float2* xg = xs + gr * kDftN;
  float2 v[R1];
  for (int i = 0; i < R1; ++i) v[i] = src[t + R2 * i];
  fft_pass1<kDftN, INV>(v, t, tw);
  for (int k1 = 0; k1 < R1; ++k1) xg[k1 * R2 + (t ^ (k1 & (R2 - 1)))] = v[p1_index<kDftN>(k1)];
  __syncwarp();
  for (int tt = 0; tt < R2; ++tt) v[tt] = xg[t * R2 + (tt ^ t)];
  fft_pass2<kDftN, INV>(v);
  for (int k2 = 0; k2 < R2; ++k2) zs[(t + R1 * k2) * kZsPad + gr] = v[p2_index<kDftN>(0, k2)];
  __syncthreads();
  float2* dst = out + (size_t)f * kDftN * kDftN + r0;
  for (int i = threadIdx.x; i < kTileElems; i += kThreads) {
    const int k = i / kDftRows, r = i % kDftRows;
    dst[(size_t)k * kDftN + r] = zs[k * kZsPad + r];
  }
}

// Fills the device tables (once per device, before any capture) and sets the
// kernels' shared-memory limit.
cudaError_t prepare_dft256(cudaStream_t s) {
  const void* fs[4] = {(const void*)k_dft256_rows_tc<false>, (const void*)k_dft256_rows_tc<true>,
                       (const void*)k_dft256_rows_fp32<false>, (const void*)k_dft256_rows_fp32<true>};
  for (int i = 0; i < 4; ++i) {
    const cudaError_t e = cudaFuncSetAttribute(fs[i], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)(i < 2 ? kDftTcSmem : kDftSmem));
    if (e != cudaSuccess) return e;
  }
  k_dft_tables<<<1, kDftN, 0, s>>>();
  return cudaGetLastError();
}

cudaError_t launch_dft256(const float2* in, float2* work, float2* out, int frames, bool inverse, int precision,
                          cudaStream_t s) {
  const int blocks = frames * (kDftN / kDftRows);
  for (int pass = 0; pass < 2; ++pass) {
    const float2* a = pass == 0 ? in : work;
    float2* b = pass == 0 ? work : out;
    if (precision == 1) {
      if (inverse) k_dft256_rows_tc<true><<<blocks, kThreads, kDftTcSmem, s>>>(a, b);
      else k_dft256_rows_tc<false><<<blocks, kThreads, kDftTcSmem, s>>>(a, b);
    } else {
      if (inverse) k_dft256_rows_fp32<true><<<blocks, kThreads, kDftSmem, s>>>(a, b);
      else k_dft256_rows_fp32<false><<<blocks, kThreads, kDftSmem, s>>>(a, b);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace dmk

extern "C" int dm_dft2(const float* in, float* work, float* out, int32_t n, int32_t frames, int32_t inverse,
                       int32_t precision, void* stream) {
  using namespace dmk;
  if (n != kDftN) { set_global_error("dm_dft2: n must be 256"); return DM_EINVAL; }
  if (frames < 1 || (long long)frames * kDftN * kDftN >= (1ll << 40)) {
    set_global_error("dm_dft2: frames out of range");
    return DM_EINVAL;
  }
  if (!in || !work || !out) { set_global_error("dm_dft2: a pointer is NULL"); return DM_EINVAL; }
  if (precision != DM_DFT_FP32 && precision != DM_DFT_BF16X3 && precision != DM_DFT_BF16X3_TC05) {
    set_global_error("dm_dft2: unknown precision");
    return DM_EINVAL;
  }
  if (work == in || work == out) { set_global_error("dm_dft2: work must not alias in or out"); return DM_EINVAL; }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  static std::mutex mu;
  static bool ready[64] = {}, ready_tc[64] = {};
  if (e == cudaSuccess && (dev < 0 || dev >= 64)) e = cudaErrorInvalidDevice;
  if (e == cudaSuccess) {
    std::lock_guard<std::mutex> lock(mu);
    if (!ready[dev]) {
      e = prepare_dft256(static_cast<cudaStream_t>(stream));
      if (e == cudaSuccess) ready[dev] = true;
    }
    if (e == cudaSuccess && precision == DM_DFT_BF16X3_TC05 && !ready_tc[dev]) {
      e = prepare_dft256_tc05(static_cast<cudaStream_t>(stream));
      if (e == cudaSuccess) ready_tc[dev] = true;
    }
  }
  if (e == cudaSuccess && precision == DM_DFT_BF16X3_TC05)
    e = launch_dft256_tc05(reinterpret_cast<const float2*>(in), reinterpret_cast<float2*>(work),
                           reinterpret_cast<float2*>(out), frames, inverse != 0, static_cast<cudaStream_t>(stream));
  else if (e == cudaSuccess)
    e = launch_dft256(reinterpret_cast<const float2*>(in), reinterpret_cast<float2*>(work),
                      reinterpret_cast<float2*>(out), frames, inverse != 0, precision,
                      static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    set_global_error(cudaGetErrorString(e));
    return DM_ECUDA;
  }
  return DM_OK;
}

extern "C" int dm_dft2_check(void) {
  int timed_out = 0;
  const cudaError_t e = dmk::dft256_tc05_status(&timed_out);
  if (e != cudaSuccess) {
    dmk::set_global_error(cudaGetErrorString(e));
    return DM_ECUDA;
  }
  if (timed_out) {
    dmk::set_global_error("dm_dft2: a bounded wait of the tcgen05 form gave up");
    return DM_ETIMEOUT;
  }
  return DM_OK;
}
