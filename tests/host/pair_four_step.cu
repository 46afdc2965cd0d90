// Host-side check of the decomposition behind the warp-pair row transform (3840-wide rows:
// M = 1920 = 64 x 30 complex points), built from the same register codelets (ils_dft.cuh):
//   1. for each g < 64: the 30-point DFT of x[g + 64 n2] over n2, times w_M^{g k2} taken from a
//      64-wide four-step table laid out as twW[W + 64 k2 + g] = w_W^{2 g k2 mod W};
//   2. for each k2 < 30 and h in {0, 1}: the 32-point DFT Z_h of the stride-2 half y[h + 2 b] of
//      the 64 values of index k2, Z_1 times w_64^k (the compile-time twiddle of the codelets);
//   3. the radix-2 join X[k2 + 30 (k + 32 c)] = Z_0[k] + (-1)^c w_64^k Z_1[k].
// Prints "direction max_rel_err" for the forward and the inverse transform against a
// brute-force DFT in double precision.  Built and run by tests/test_codelets_host.py.
#include <cmath>
#include <cstdio>
#include <vector>

#include "ils_dft.cuh"

constexpr int L = 30, M = 64 * L, W = 2 * M;

template <bool INV>
double check() {
  std::vector<float2> x(M), roots(W), ft(M), X(M);
  unsigned s = 987654321u + (INV ? 11u : 0u);
  for (int n = 0; n < M; ++n) {
    s = s * 1664525u + 1013904223u;
    const float re = (float)((double)(s >> 8) / 16777216.0 - 0.5);
    s = s * 1664525u + 1013904223u;
    const float im = (float)((double)(s >> 8) / 16777216.0 - 0.5);
    x[n] = ils::c2(re, im);
  }
  for (int t = 0; t < W; ++t) {
    const double a = -2.0 * M_PI * (double)t / (double)W;
    roots[t] = ils::c2((float)std::cos(a), (float)std::sin(a));
  }
  for (int t = 0; t < M; ++t) ft[t] = roots[(2 * (t % 64) * (t / 64)) % W];  // k2-major, 64 wide
  // step 1: lines[k2][g]
  std::vector<float2> lines((size_t)L * 64);
  for (int g = 0; g < 64; ++g) {
    float2 v[L];
    for (int n2 = 0; n2 < L; ++n2) v[n2] = x[g + 64 * n2];
    ils::dft_reg<L, INV>(v);
    for (int k2 = 1; k2 < L; ++k2) {
      float2 w = ft[64 * k2 + g];
      if (INV) w.y = -w.y;
      v[k2] = ils::cmul(v[k2], w);
    }
    for (int k2 = 0; k2 < L; ++k2) lines[(size_t)k2 * 64 + g] = v[k2];
  }
  // steps 2 and 3
  constexpr ils::Roots<64> w64{};
  for (int k2 = 0; k2 < L; ++k2) {
    float2 z[2][32];
    for (int h = 0; h < 2; ++h) {
      for (int b = 0; b < 32; ++b) z[h][b] = lines[(size_t)k2 * 64 + h + 2 * b];
      ils::dft_reg<32, INV>(z[h]);
    }
    for (int k = 1; k < 32; ++k) z[1][k] = ils::twiddle_const<64, INV>(z[1][k], k, w64);
    for (int k = 0; k < 32; ++k) {
      X[k2 + L * k] = ils::cadd(z[0][k], z[1][k]);
      X[k2 + L * (k + 32)] = ils::csub(z[0][k], z[1][k]);
    }
  }
  double err = 0.0, mag = 0.0;
  const double sg = INV ? 1.0 : -1.0;
  for (int k = 0; k < M; ++k) {
    double re = 0.0, im = 0.0;
    for (int n = 0; n < M; ++n) {
      const double a = sg * 2.0 * M_PI * (double)((long)n * k % M) / M;
      re += x[n].x * std::cos(a) - x[n].y * std::sin(a);
      im += x[n].x * std::sin(a) + x[n].y * std::cos(a);
    }
    err = std::fmax(err, std::hypot(re - X[k].x, im - X[k].y));
    mag = std::fmax(mag, std::hypot(re, im));
  }
  return err / mag;
}

int main() {
  std::printf("forward %.3e\ninverse %.3e\n", check<false>(), check<true>());
  return 0;
}
