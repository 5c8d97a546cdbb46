// Register-level FFT building blocks for the difference-map Fourier step.
//
// A length-N transform (N = R1 * R2, a power of two) is computed by a group
// of R2 threads that each hold R1 complex values:
//   pass 1: thread t transforms x[t + R2*i], i < R1, in registers (an R1-point
//           DFT), then multiplies output k1 by W_N^(t*k1);
//   exchange through a small shared buffer laid out [k1][t] with one float2
//           of padding per row (bank-conflict free for both access patterns);
//   pass 2: thread t' transforms, for each k1 = t' + R2*d (d < R1/R2), the R2
//           values over t, producing X[k1 + R1*k2].
// This is the Cooley-Tukey split X[k1 + R1 k2] =
//   sum_t W_R2^(t k2) W_N^(t k1) sum_i x[t + R2 i] W_R1^(i k1).
//
// Everything here is __host__ __device__ so that the host test harness can
// run the same code on the CPU.  Sign convention: forward uses
// W = exp(-2 pi i / n); inverse uses the conjugate and is unnormalised.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#ifndef DM_HD
#define DM_HD __host__ __device__ __forceinline__
#endif

namespace dmk {

// Complex add/sub.  On sm_100+ devices a single packed f32x2 instruction does
// both halves (each half is an ordinary round-to-nearest FP32 add).
DM_HD float2 cadd(float2 a, float2 b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r)
      : "l"(*reinterpret_cast<const unsigned long long*>(&a)), "l"(*reinterpret_cast<const unsigned long long*>(&b)));
  return *reinterpret_cast<float2*>(&r);
#else
  return make_float2(a.x + b.x, a.y + b.y);
#endif
}
DM_HD float2 csub(float2 a, float2 b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r)
      : "l"(*reinterpret_cast<const unsigned long long*>(&a)), "l"(*reinterpret_cast<const unsigned long long*>(&b)));
  return *reinterpret_cast<float2*>(&r);
#else
  return make_float2(a.x - b.x, a.y - b.y);
#endif
}
DM_HD float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// a * b
DM_HD float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// conj(a) * b
DM_HD float2 cconjmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
// a * conj(b) when INV, a * b otherwise (b is a forward twiddle)
template <bool INV>
DM_HD float2 ctw(float2 a, float2 b) {
  return INV ? make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y)) : cmul(a, b);
}
DM_HD float cnorm(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

// cos(pi/8), sin(pi/8), sqrt(1/2)
#define DM_C8 0.92387953251128674f
#define DM_S8 0.38268343236508977f
#define DM_R2 0.70710678118654752f

// a * exp(-+2 pi i m / 16): '-' for the forward transform, '+' for INV.
// m is a compile-time constant after unrolling, so the switch folds away.
template <bool INV>
DM_HD float2 mul_w16(float2 a, int m) {
  m &= 15;
  float2 r;
  switch (m & 7) {
    case 0: r = a; break;
    case 1: r = INV ? cmul(a, make_float2(DM_C8, DM_S8)) : cmul(a, make_float2(DM_C8, -DM_S8)); break;
    case 2: r = INV ? make_float2(DM_R2 * (a.x - a.y), DM_R2 * (a.x + a.y))
                    : make_float2(DM_R2 * (a.x + a.y), DM_R2 * (a.y - a.x)); break;
    case 3: r = INV ? cmul(a, make_float2(DM_S8, DM_C8)) : cmul(a, make_float2(DM_S8, -DM_C8)); break;
    case 4: r = INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x); break;
    case 5: r = INV ? cmul(a, make_float2(-DM_S8, DM_C8)) : cmul(a, make_float2(-DM_S8, -DM_C8)); break;
    case 6: r = INV ? make_float2(-DM_R2 * (a.x + a.y), DM_R2 * (a.x - a.y))
                    : make_float2(DM_R2 * (a.y - a.x), -DM_R2 * (a.x + a.y)); break;
    default: r = INV ? cmul(a, make_float2(-DM_C8, DM_S8)) : cmul(a, make_float2(-DM_C8, -DM_S8)); break;
  }
  if (m & 8) r = make_float2(-r.x, -r.y);
  return r;
}

template <int R>
struct Log2 { static constexpr int v = 1 + Log2<R / 2>::v; };
template <>
struct Log2<1> { static constexpr int v = 0; };

template <int R>
DM_HD constexpr int bitrev(int k) {
  int r = 0;
  for (int b = 0; b < Log2<R>::v; ++b) r |= ((k >> b) & 1) << (Log2<R>::v - 1 - b);
  return r;
}

// In-register R-point DFT (R in {2,4,8,16}) of v[0..R), radix-2 decimation
// in frequency.  On return v[bitrev<R>(k)] holds X[k].
template <int R, bool INV>
DM_HD void dft_reg(float2* v) {
#pragma unroll
  for (int half = R / 2; half >= 1; half >>= 1) {
#pragma unroll
    for (int b = 0; b < R; b += 2 * half) {
#pragma unroll
      for (int i = 0; i < half; ++i) {
        const float2 a = v[b + i];
        const float2 c = v[b + i + half];
        v[b + i] = cadd(a, c);
        v[b + i + half] = mul_w16<INV>(csub(a, c), i * (16 / (2 * half)));
      }
    }
  }
}

// Split of N into R1 (values per thread) x R2 (threads per transform).
template <int N> struct FftShape;
template <> struct FftShape<16>  { static constexpr int R1 = 4,  R2 = 4;  };
template <> struct FftShape<32>  { static constexpr int R1 = 8,  R2 = 4;  };
template <> struct FftShape<64>  { static constexpr int R1 = 8,  R2 = 8;  };
template <> struct FftShape<128> { static constexpr int R1 = 16, R2 = 8;  };
template <> struct FftShape<256> { static constexpr int R1 = 16, R2 = 16; };

// Pass 1 for thread t, in place: v[i] = x[t + R2 i] on entry; on return the
// twiddled value for k1, Y_t[k1] W_N^(t k1), sits at v[p1_index(k1)].
// tw[m] = exp(-2 pi i m / N).
template <int N>
DM_HD constexpr int p1_index(int k1) { return bitrev<FftShape<N>::R1>(k1); }

template <int N, bool INV>
DM_HD void fft_pass1(float2 (&v)[FftShape<N>::R1], int t, const float2* tw) {
  constexpr int R1 = FftShape<N>::R1;
  dft_reg<R1, INV>(v);
#pragma unroll
  for (int k1 = 1; k1 < R1; ++k1) v[bitrev<R1>(k1)] = ctw<INV>(v[bitrev<R1>(k1)], tw[t * k1]);
}

// Pass 2 for thread t', in place: u[d*R2 + t] = Y_t[k1 = t' + R2 d] on entry
// (t < R2, d < R1/R2); on return X[k1 + R1 k2] sits at u[p2_index(d, k2)].
template <int N>
DM_HD constexpr int p2_index(int d, int k2) { return d * FftShape<N>::R2 + bitrev<FftShape<N>::R2>(k2); }

template <int N, bool INV>
DM_HD void fft_pass2(float2 (&u)[FftShape<N>::R1]) {
  constexpr int R1 = FftShape<N>::R1, R2 = FftShape<N>::R2, D = R1 / R2;
#pragma unroll
  for (int d = 0; d < D; ++d) dft_reg<R2, INV>(u + d * R2);
}

}  // namespace dmk
