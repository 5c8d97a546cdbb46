// Host-side check of the register FFT building blocks used by the CUDA
// Fourier step: the two-pass split (pass 1, shared exchange, pass 2) is run
// on the CPU with the threads emulated in loops and compared with a direct
// O(N^2) DFT in double precision.  Prints the worst relative error per N and
// exits non-zero if any exceeds the bound given on the command line.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "../../paper_1808_10375_gb300/csrc/dm_fft.cuh"

using namespace dmk;

template <int N, bool INV>
static double check(std::mt19937_64& rng) {
  constexpr int R1 = FftShape<N>::R1, R2 = FftShape<N>::R2, D = R1 / R2;
  std::normal_distribution<double> nd;
  std::vector<float2> x(N), tw(tw_entries<N>());
  for (int i = 0; i < N; ++i) x[i] = make_float2((float)nd(rng), (float)nd(rng));
  tw_fill<N>(tw.data(), [](int m) {
    const double a = -2.0 * M_PI * m / N;
    return make_float2((float)std::cos(a), (float)std::sin(a));
  });
  // pass 1 per thread, exchange buffer [k1][t]
  std::vector<float2> xb(R1 * R2);
  for (int t = 0; t < R2; ++t) {
    float2 v[R1];
    for (int i = 0; i < R1; ++i) v[i] = x[t + R2 * i];
    fft_pass1<N, INV>(v, t, tw.data());
    for (int k1 = 0; k1 < R1; ++k1) xb[k1 * R2 + t] = v[p1_index<N>(k1)];
  }
  std::vector<float2> X(N);
  for (int tp = 0; tp < R2; ++tp) {
    float2 u[R1];
    for (int d = 0; d < D; ++d)
      for (int t = 0; t < R2; ++t) u[d * R2 + t] = xb[(tp + R2 * d) * R2 + t];
    fft_pass2<N, INV>(u);
    for (int d = 0; d < D; ++d)
      for (int k2 = 0; k2 < R2; ++k2) X[tp + R2 * d + R1 * k2] = u[p2_index<N>(d, k2)];
  }
  double num = 0, den = 0;
  const double sg = INV ? 1.0 : -1.0;
  for (int k = 0; k < N; ++k) {
    double re = 0, im = 0;
    for (int n = 0; n < N; ++n) {
      const double a = sg * 2.0 * M_PI * (double)((long)n * k % N) / N;
      re += x[n].x * std::cos(a) - x[n].y * std::sin(a);
      im += x[n].x * std::sin(a) + x[n].y * std::cos(a);
    }
    num += (X[k].x - re) * (X[k].x - re) + (X[k].y - im) * (X[k].y - im);
    den += re * re + im * im;
  }
  return std::sqrt(num / den);
}

// Inverse transform started from the pass-2 distribution (ifft_stepA, an
// exchange, ifft_stepB) against the direct inverse DFT.
template <int N>
static double check_dif(std::mt19937_64& rng) {
  constexpr int R1 = FftShape<N>::R1, R2 = FftShape<N>::R2, D = R1 / R2;
  std::normal_distribution<double> nd;
  std::vector<float2> X(N), tw(tw_entries<N>());
  for (int i = 0; i < N; ++i) X[i] = make_float2((float)nd(rng), (float)nd(rng));
  tw_fill<N>(tw.data(), [](int m) {
    const double a = -2.0 * M_PI * m / N;
    return make_float2((float)std::cos(a), (float)std::sin(a));
  });
  std::vector<float2> xb(R1 * R2);  // [k1][t]
  for (int tp = 0; tp < R2; ++tp) {
    float2 u[R1];
    for (int d = 0; d < D; ++d)
      for (int k2 = 0; k2 < R2; ++k2) u[p2_index<N>(d, k2)] = X[tp + R2 * d + R1 * k2];
    ifft_stepA<N>(u, tp, tw_dif<N>(tw.data()));
    for (int d = 0; d < D; ++d)
      for (int t = 0; t < R2; ++t) xb[(tp + R2 * d) * R2 + t] = u[d * R2 + t];
  }
  std::vector<float2> x(N);
  for (int t = 0; t < R2; ++t) {
    float2 v[R1];
    for (int k1 = 0; k1 < R1; ++k1) v[k1] = xb[k1 * R2 + t];
    ifft_stepB<N>(v);
    for (int i = 0; i < R1; ++i) x[t + R2 * i] = v[p1_index<N>(i)];
  }
  double num = 0, den = 0;
  for (int n = 0; n < N; ++n) {
    double re = 0, im = 0;
    for (int k = 0; k < N; ++k) {
      const double a = 2.0 * M_PI * (double)((long)n * k % N) / N;
      re += X[k].x * std::cos(a) - X[k].y * std::sin(a);
      im += X[k].x * std::sin(a) + X[k].y * std::cos(a);
    }
    num += (x[n].x - re) * (x[n].x - re) + (x[n].y - im) * (x[n].y - im);
    den += re * re + im * im;
  }
  return std::sqrt(num / den);
}

template <int R, bool INV>
static double check_reg(std::mt19937_64& rng) {
  std::normal_distribution<double> nd;
  float2 v[R], x[R];
  for (int i = 0; i < R; ++i) x[i] = v[i] = make_float2((float)nd(rng), (float)nd(rng));
  dft_reg<R, INV>(v);
  double num = 0, den = 0;
  const double sg = INV ? 1.0 : -1.0;
  for (int k = 0; k < R; ++k) {
    double re = 0, im = 0;
    for (int n = 0; n < R; ++n) {
      const double a = sg * 2.0 * M_PI * n * k / R;
      re += x[n].x * std::cos(a) - x[n].y * std::sin(a);
      im += x[n].x * std::sin(a) + x[n].y * std::cos(a);
    }
    const float2 g = v[out_index<R>(k)];
    num += (g.x - re) * (g.x - re) + (g.y - im) * (g.y - im);
    den += re * re + im * im;
  }
  return std::sqrt(num / den);
}

int main(int argc, char** argv) {
  const double bound = argc > 1 ? std::atof(argv[1]) : 1e-6;
  std::mt19937_64 rng(12345);
  double worst = 0;
  auto rep = [&](const char* what, int n, double e) {
    std::printf("%s %d %.3e\n", what, n, e);
    if (e > worst) worst = e;
  };
  for (int rep_i = 0; rep_i < 4; ++rep_i) {
    rep("reg_fwd", 2, check_reg<2, false>(rng));   rep("reg_inv", 2, check_reg<2, true>(rng));
    rep("reg_fwd", 4, check_reg<4, false>(rng));   rep("reg_inv", 4, check_reg<4, true>(rng));
    rep("reg_fwd", 8, check_reg<8, false>(rng));   rep("reg_inv", 8, check_reg<8, true>(rng));
    rep("reg_fwd", 16, check_reg<16, false>(rng)); rep("reg_inv", 16, check_reg<16, true>(rng));
    rep("fft_fwd", 16, check<16, false>(rng));   rep("fft_inv", 16, check<16, true>(rng));
    rep("fft_fwd", 32, check<32, false>(rng));   rep("fft_inv", 32, check<32, true>(rng));
    rep("fft_fwd", 64, check<64, false>(rng));   rep("fft_inv", 64, check<64, true>(rng));
    rep("fft_fwd", 128, check<128, false>(rng)); rep("fft_inv", 128, check<128, true>(rng));
    rep("fft_fwd", 256, check<256, false>(rng)); rep("fft_inv", 256, check<256, true>(rng));
    rep("ifft_dif", 16, check_dif<16>(rng));   rep("ifft_dif", 32, check_dif<32>(rng));
    rep("ifft_dif", 64, check_dif<64>(rng));   rep("ifft_dif", 128, check_dif<128>(rng));
    rep("ifft_dif", 256, check_dif<256>(rng));
  }
  std::printf("worst %.3e bound %.1e\n", worst, bound);
  return worst <= bound ? 0 : 1;
}
