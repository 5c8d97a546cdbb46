// Register-level FFT building blocks for the difference-map Fourier step.
//
// A length-N transform (N = R1 * R2, a power of two) is computed by a group
// of R2 threads that each hold R1 complex values:
//   pass 1: thread t transforms x[t + R2*i], i < R1, in registers (an R1-point
//           DFT), then multiplies output k1 by W_N^(t*k1) (table twF, below);
//   exchange through a small shared buffer laid out [k1][t ^ (k1 mod R2)]
//           (the XOR swizzle keeps both access patterns bank-conflict free);
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

// Complex add/sub.  On sm_100+ devices one packed f32x2 instruction does both
// halves (each half is an ordinary round-to-nearest FP32 add).
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


// Radix-4 butterfly in place (forward: y_k = sum_n a_n (-i)^(nk); INV uses
// +i).  The multiplication by -+i is folded into the final adds.
template <bool INV>
DM_HD void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  const float2 t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), d = csub(a1, a3);
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  if (!INV) {
    a1 = make_float2(t1.x + d.y, t1.y - d.x);
    a3 = make_float2(t1.x - d.y, t1.y + d.x);
  } else {
    a1 = make_float2(t1.x - d.y, t1.y + d.x);
    a3 = make_float2(t1.x + d.y, t1.y - d.x);
  }
}

// In-register R-point DFT (R in {2, 4, 8, 16}) of v[0..R).  On return
// v[out_index<R>(k)] holds X[k].
//   R = 16: 4 x 4 split, X[k1 + 4 k2] at v[4 k1 + k2];
//   R = 8:  2 x 4 split, X[k1 + 4 k2] at v[2 k1 + k2];
//   R = 4, 2: natural order.
template <int R, bool INV>
DM_HD void dft_reg(float2* v) {
  if constexpr (R == 2) {
    const float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  } else if constexpr (R == 4) {
    dft4<INV>(v[0], v[1], v[2], v[3]);
  } else if constexpr (R == 8) {
    // n = 2 n1 + n2: DFT4 over n1 for each n2, twiddle W8^(n2 k1), DFT2 over n2
    dft4<INV>(v[0], v[2], v[4], v[6]);
    dft4<INV>(v[1], v[3], v[5], v[7]);
    v[3] = mul_w16<INV>(v[3], 2);
    v[5] = mul_w16<INV>(v[5], 4);
    v[7] = mul_w16<INV>(v[7], 6);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      const float2 a = v[2 * k1], b = v[2 * k1 + 1];
      v[2 * k1] = cadd(a, b);
      v[2 * k1 + 1] = csub(a, b);
    }
  } else {
    // n = 4 n1 + n2: DFT4 over n1 for each n2, twiddle W16^(n2 k1), DFT4 over n2
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4<INV>(v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]);
    v[5] = mul_w16<INV>(v[5], 1);
    v[9] = mul_w16<INV>(v[9], 2);
    v[13] = mul_w16<INV>(v[13], 3);
    v[6] = mul_w16<INV>(v[6], 2);
    v[10] = mul_w16<INV>(v[10], 4);
    v[14] = mul_w16<INV>(v[14], 6);
    v[7] = mul_w16<INV>(v[7], 3);
    v[11] = mul_w16<INV>(v[11], 6);
    v[15] = mul_w16<INV>(v[15], 9);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4<INV>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
  }
}

template <int R>
DM_HD constexpr int out_index(int k) {
  return R == 16 ? 4 * (k & 3) + (k >> 2) : R == 8 ? 2 * (k & 3) + (k >> 2) : k;
}

// Split of N into R1 (values per thread) x R2 (threads per transform).
template <int N> struct FftShape;
template <> struct FftShape<16>  { static constexpr int R1 = 4,  R2 = 4;  };
template <> struct FftShape<32>  { static constexpr int R1 = 8,  R2 = 4;  };
template <> struct FftShape<64>  { static constexpr int R1 = 8,  R2 = 8;  };
template <> struct FftShape<128> { static constexpr int R1 = 16, R2 = 8;  };
template <> struct FftShape<256> { static constexpr int R1 = 16, R2 = 16; };

// Twiddle tables, both holding W_N^(t k1) = exp(-2 pi i t k1 / N):
//   twF[k1 * R2 + t] (k1 < R1, t < R2): pass 1, where thread t reads one row
//       per k1 (consecutive threads, consecutive entries);
//   twD[t * R1 + k1]: the inverse that starts from the pass-2 distribution
//       (below), where the thread holding k1 reads one entry per t.
// When R1 == R2 the two tables coincide (W is symmetric in t and k1) and only
// twF is stored; otherwise twD follows twF.  tw_entries<N>() is the total.
template <int N>
DM_HD constexpr int tw_entries() { return FftShape<N>::R1 == FftShape<N>::R2 ? N : 2 * N; }

template <int N>
DM_HD const float2* tw_dif(const float2* twF) { return FftShape<N>::R1 == FftShape<N>::R2 ? twF : twF + N; }

// Host side: fill the tables from w(m) = W_N^m (computed in double precision).
template <int N, class F>
inline void tw_fill(float2* tab, F w) {
  constexpr int R1 = FftShape<N>::R1, R2 = FftShape<N>::R2;
  for (int k1 = 0; k1 < R1; ++k1)
    for (int t = 0; t < R2; ++t) tab[k1 * R2 + t] = w((t * k1) % N);
  if (R1 != R2)
    for (int t = 0; t < R2; ++t)
      for (int k1 = 0; k1 < R1; ++k1) tab[N + t * R1 + k1] = w((t * k1) % N);
}

// Pass 1 for thread t, in place: v[i] = x[t + R2 i] on entry; on return the
// twiddled value for k1, Y_t[k1] W_N^(t k1), sits at v[p1_index(k1)].
template <int N>
DM_HD constexpr int p1_index(int k1) { return out_index<FftShape<N>::R1>(k1); }

template <int N, bool INV>
DM_HD void fft_pass1(float2 (&v)[FftShape<N>::R1], int t, const float2* twF) {
  constexpr int R1 = FftShape<N>::R1, R2 = FftShape<N>::R2;
  dft_reg<R1, INV>(v);
#pragma unroll
  for (int k1 = 1; k1 < R1; ++k1) v[out_index<R1>(k1)] = ctw<INV>(v[out_index<R1>(k1)], twF[k1 * R2 + t]);
}

// Pass 2 for thread t', in place: u[d*R2 + t] = Y_t[k1 = t' + R2 d] on entry
// (t < R2, d < R1/R2); on return X[k1 + R1 k2] sits at u[p2_index(d, k2)].
template <int N>
DM_HD constexpr int p2_index(int d, int k2) { return d * FftShape<N>::R2 + out_index<FftShape<N>::R2>(k2); }

template <int N, bool INV>
DM_HD void fft_pass2(float2 (&u)[FftShape<N>::R1]) {
  constexpr int R1 = FftShape<N>::R1, R2 = FftShape<N>::R2, D = R1 / R2;
#pragma unroll
  for (int d = 0; d < D; ++d) dft_reg<R2, INV>(u + d * R2);
}

// Inverse transform taken from the pass-2 distribution (no reordering in
// between): thread t' holds X[k1 + R1 k2], k1 = t' + R2 d, at
// u[p2_index(d, k2)].  With n = t + R2 i,
//   x[n] = sum_k1 W_R1^(-i k1) W_N^(-t k1) sum_k2 X[k1 + R1 k2] W_R2^(-t k2),
// so step A (in registers) is, for each d, an R2-point inverse DFT over k2
// followed by the factor W_N^(-t k1); afterwards the value for (k1, t) sits
// at u[d * R2 + t].  After an exchange that gives thread t the values for
// every k1 (natural order, v[k1]), step B is the R1-point inverse DFT over
// k1, leaving x[t + R2 i] at v[p1_index(i)]: the distribution pass 1 reads.
template <int N>
DM_HD void ifft_stepA(float2 (&u)[FftShape<N>::R1], int tp, const float2* twD) {
  constexpr int R1 = FftShape<N>::R1, R2 = FftShape<N>::R2, D = R1 / R2;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    float2 w[R2];
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) w[k2] = u[d * R2 + out_index<R2>(k2)];
    dft_reg<R2, true>(w);
    const int k1 = tp + R2 * d;
    u[d * R2] = w[out_index<R2>(0)];
#pragma unroll
    for (int t = 1; t < R2; ++t) u[d * R2 + t] = ctw<true>(w[out_index<R2>(t)], twD[t * R1 + k1]);
  }
}

template <int N>
DM_HD void ifft_stepB(float2 (&v)[FftShape<N>::R1]) {
  dft_reg<FftShape<N>::R1, true>(v);
}

}  // namespace dmk
