// Host-side check of the register DFT codelets (ils_dft.cuh): every supported size, both
// directions, against a brute-force DFT in double precision.  Prints one line per size:
// "R max_rel_err".  Built and run by tests/test_codelets_host.py (no GPU needed).
#include <cmath>
#include <cstdio>
#include <cstdlib>

#include "ils_dft.cuh"

template <int R, bool INV>
double check() {
  float2 v[R];
  double xr[R], xi[R];
  unsigned s = 12345u + 7u * R + (INV ? 1u : 0u);
  for (int n = 0; n < R; ++n) {
    s = s * 1664525u + 1013904223u;
    xr[n] = (double)(s >> 8) / 16777216.0 - 0.5;
    s = s * 1664525u + 1013904223u;
    xi[n] = (double)(s >> 8) / 16777216.0 - 0.5;
    v[n] = ils::c2((float)xr[n], (float)xi[n]);
    xr[n] = v[n].x;
    xi[n] = v[n].y;
  }
  ils::dft_reg<R, INV>(v);
  double err = 0.0, mag = 0.0;
  const double sg = INV ? 1.0 : -1.0;
  for (int k = 0; k < R; ++k) {
    double re = 0.0, im = 0.0;
    for (int n = 0; n < R; ++n) {
      const double a = sg * 2.0 * M_PI * (double)((long)n * k % R) / R;
      re += xr[n] * std::cos(a) - xi[n] * std::sin(a);
      im += xr[n] * std::sin(a) + xi[n] * std::cos(a);
    }
    err = std::fmax(err, std::hypot(re - v[k].x, im - v[k].y));
    mag = std::fmax(mag, std::hypot(re, im));
  }
  return err / mag;
}

template <int R>
void run() {
  std::printf("%d %.3e %.3e\n", R, check<R, false>(), check<R, true>());
}

int main() {
  run<2>(); run<3>(); run<4>(); run<5>(); run<6>(); run<8>(); run<9>(); run<10>(); run<12>(); run<15>();
  run<16>(); run<20>(); run<24>(); run<25>(); run<27>(); run<30>(); run<32>(); run<36>(); run<40>();
  run<45>(); run<48>(); run<54>(); run<60>(); run<64>();
  return 0;
}
