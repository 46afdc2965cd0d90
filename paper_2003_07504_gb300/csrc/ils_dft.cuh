// Small DFTs held entirely in registers, for the FFT stages of the ILS kernels.
//
// dft_reg<R, INV>(v) replaces v[0..R-1] by its R-point DFT (forward: exp(-2 pi i jk/R),
// INV: exp(+2 pi i jk/R), unnormalized).  R in {2,3,4,5,8} are written out; every other
// supported R = A*B is split once on registers:
//  * gcd(A, B) = 1: the prime-factor (Good-Thomas) mapping.  Input n = (B n1 + A n2) mod R
//    and output k with k = k1 (mod A), k = k2 (mod B) turn the R-point DFT into B DFTs of
//    size A followed by A DFTs of size B with no twiddle multiplications at all (the
//    kernel exp(-2 pi i n k / R) factors exactly into the two smaller kernels);
//  * otherwise one Cooley-Tukey step: B DFTs of size A on the stride-B subsequences,
//    multiplication by w_R^{n2 k1}, then A DFTs of size B, with output index k1 + A k2.
//    Twiddles on the eighth turns (w = +-1, +-i, (+-1 +- i)/sqrt 2) are applied as sign
//    changes and swaps (and one sqrt(1/2) scaling); the others come from a compile-time table
//    built with a Taylor-series sine/cosine written here (no math-library call), so after
//    unrolling every twiddle is an immediate.
//
// All functions are __host__ __device__ so the same code can be exercised on the CPU.
#pragma once
#include <cuda_runtime.h>

#if defined(__CUDACC__)
#define ILS_HD __host__ __device__ __forceinline__
#else
#define ILS_HD inline
#endif

namespace ils {

ILS_HD float2 c2(float x, float y) { float2 r; r.x = x; r.y = y; return r; }
ILS_HD float2 cadd(float2 a, float2 b) { return c2(a.x + b.x, a.y + b.y); }
ILS_HD float2 csub(float2 a, float2 b) { return c2(a.x - b.x, a.y - b.y); }
ILS_HD float2 cmul(float2 a, float2 b) { return c2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
ILS_HD float2 cconj(float2 a) { return c2(a.x, -a.y); }
ILS_HD float2 cscale(float2 a, float s) { return c2(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <bool INV>
ILS_HD float2 rot90(float2 a) {
  return INV ? c2(-a.y, a.x) : c2(a.y, -a.x);
}

// ---------------------------------------------------------------- compile-time roots of unity
// theta = 2 pi m / R is reduced exactly on the integer grid to [-pi, pi]; there the Taylor
// series with 20 terms is accurate to well below double rounding.
constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr double ct_theta(long m, long R) {
  long r = m % R;
  if (r < 0) r += R;
  if (2 * r > R) r -= R;
  return 2.0 * kPi * (double)r / (double)R;
}
constexpr double ct_sin(double x) {
  double term = x, sum = x;
  for (int n = 1; n < 20; ++n) {
    term *= -x * x / ((2.0 * n) * (2.0 * n + 1.0));
    sum += term;
  }
  return sum;
}
constexpr double ct_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int n = 1; n < 20; ++n) {
    term *= -x * x / ((2.0 * n - 1.0) * (2.0 * n));
    sum += term;
  }
  return sum;
}
// exp(-2 pi i m / R) (forward root) as a float2 constant
template <int R>
struct Roots {
  float re[R], im[R];
  constexpr Roots() : re(), im() {
    for (int m = 0; m < R; ++m) {
      re[m] = (float)ct_cos(ct_theta(m, R));
      im[m] = (float)(-ct_sin(ct_theta(m, R)));
    }
  }
};

// ---------------------------------------------------------------- written-out small DFTs

template <bool INV>
ILS_HD void dft2(float2* v) {
  float2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <bool INV>
ILS_HD void dft4(float2* v) {
  float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
  float2 s13 = cadd(v[1], v[3]), d13 = rot90<INV>(csub(v[1], v[3]));
  v[0] = cadd(s02, s13);
  v[2] = csub(s02, s13);
  v[1] = cadd(d02, d13);
  v[3] = csub(d02, d13);
}

template <bool INV>
ILS_HD void dft8(float2* v) {
  constexpr float h = 0.70710678118654752440f;  // sqrt(2)/2
  float2 e[4] = {v[0], v[2], v[4], v[6]};
  float2 o[4] = {v[1], v[3], v[5], v[7]};
  dft4<INV>(e);
  dft4<INV>(o);
  // o[k] *= w_8^k
  o[1] = INV ? c2(h * (o[1].x - o[1].y), h * (o[1].x + o[1].y)) : c2(h * (o[1].x + o[1].y), h * (o[1].y - o[1].x));
  o[2] = rot90<INV>(o[2]);
  o[3] = INV ? c2(-h * (o[3].x + o[3].y), h * (o[3].x - o[3].y)) : c2(h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y));
  for (int k = 0; k < 4; ++k) {
    v[k] = cadd(e[k], o[k]);
    v[k + 4] = csub(e[k], o[k]);
  }
}

template <bool INV>
ILS_HD void dft3(float2* v) {
  constexpr float s3 = 0.86602540378443864676f;  // sin(2 pi / 3)
  float2 t = cadd(v[1], v[2]);
  float2 d = csub(v[1], v[2]);
  float2 m = c2(v[0].x - 0.5f * t.x, v[0].y - 0.5f * t.y);
  float2 r = rot90<INV>(cscale(d, s3));
  v[0] = cadd(v[0], t);
  v[1] = cadd(m, r);
  v[2] = csub(m, r);
}

template <bool INV>
ILS_HD void dft5(float2* v) {
  constexpr float c1 = 0.30901699437494742410f;   // cos(2 pi / 5)
  constexpr float c2_ = -0.80901699437494742410f; // cos(4 pi / 5)
  constexpr float s1 = 0.95105651629515357212f;   // sin(2 pi / 5)
  constexpr float s2 = 0.58778525229247312917f;   // sin(4 pi / 5)
  float2 a14 = cadd(v[1], v[4]), d14 = csub(v[1], v[4]);
  float2 a23 = cadd(v[2], v[3]), d23 = csub(v[2], v[3]);
  float2 p1 = c2(v[0].x + c1 * a14.x + c2_ * a23.x, v[0].y + c1 * a14.y + c2_ * a23.y);
  float2 p2 = c2(v[0].x + c2_ * a14.x + c1 * a23.x, v[0].y + c2_ * a14.y + c1 * a23.y);
  float2 q1 = rot90<INV>(c2(s1 * d14.x + s2 * d23.x, s1 * d14.y + s2 * d23.y));
  float2 q2 = rot90<INV>(c2(s2 * d14.x - s1 * d23.x, s2 * d14.y - s1 * d23.y));
  v[0] = c2(v[0].x + a14.x + a23.x, v[0].y + a14.y + a23.y);
  v[1] = cadd(p1, q1);
  v[4] = csub(p1, q1);
  v[2] = cadd(p2, q2);
  v[3] = csub(p2, q2);
}

// ---------------------------------------------------------------- composite sizes

template <int R>
struct Split;  // R = A * B with A the first factor used
template <> struct Split<6> { static constexpr int A = 2, B = 3; };
template <> struct Split<9> { static constexpr int A = 3, B = 3; };
template <> struct Split<10> { static constexpr int A = 2, B = 5; };
template <> struct Split<12> { static constexpr int A = 4, B = 3; };
template <> struct Split<15> { static constexpr int A = 3, B = 5; };
template <> struct Split<16> { static constexpr int A = 4, B = 4; };
template <> struct Split<20> { static constexpr int A = 4, B = 5; };
template <> struct Split<24> { static constexpr int A = 8, B = 3; };
template <> struct Split<25> { static constexpr int A = 5, B = 5; };
template <> struct Split<27> { static constexpr int A = 3, B = 9; };
template <> struct Split<30> { static constexpr int A = 2, B = 15; };
template <> struct Split<32> { static constexpr int A = 4, B = 8; };
template <> struct Split<36> { static constexpr int A = 4, B = 9; };
template <> struct Split<40> { static constexpr int A = 8, B = 5; };
template <> struct Split<45> { static constexpr int A = 5, B = 9; };
template <> struct Split<48> { static constexpr int A = 16, B = 3; };
template <> struct Split<54> { static constexpr int A = 6, B = 9; };
template <> struct Split<60> { static constexpr int A = 4, B = 15; };
template <> struct Split<64> { static constexpr int A = 8, B = 8; };

template <int R, bool INV>
ILS_HD void dft_reg(float2* v);

constexpr int ct_gcd(int a, int b) { return b == 0 ? a : ct_gcd(b, a % b); }
// x with x * a = 1 (mod m), for gcd(a, m) = 1
constexpr int ct_modinv(int a, int m) {
  for (int x = 1; x < m; ++x)
    if ((x * a) % m == 1) return x;
  return m == 1 ? 0 : -1;
}

// t * w_R^m (forward: exp(-2 pi i m / R); INV: the conjugate), m a compile-time constant after
// unrolling.  Eighth turns are exact sign changes and swaps.
template <int R, bool INV>
ILS_HD float2 twiddle_const(float2 t, int m, const Roots<R>& w) {
  constexpr float h = 0.70710678118654752440f;  // sqrt(2)/2
  m %= R;
  if (m == 0) return t;
  if ((8 * m) % R == 0) {
    const int q = 8 * m / R;  // forward angle -q pi / 4
    switch (q) {
      case 2: return rot90<INV>(t);
      case 4: return c2(-t.x, -t.y);
      case 6: return rot90<!INV>(t);
      case 1: return INV ? c2(h * (t.x - t.y), h * (t.x + t.y)) : c2(h * (t.x + t.y), h * (t.y - t.x));
      case 3: return INV ? c2(-h * (t.x + t.y), h * (t.x - t.y)) : c2(h * (t.y - t.x), -h * (t.x + t.y));
      case 5: return INV ? c2(h * (t.y - t.x), -h * (t.x + t.y)) : c2(-h * (t.x + t.y), h * (t.x - t.y));
      default: return INV ? c2(h * (t.x + t.y), h * (t.y - t.x)) : c2(h * (t.x - t.y), h * (t.x + t.y));
    }
  }
  return cmul(t, c2(w.re[m], INV ? -w.im[m] : w.im[m]));
}

template <int A, int B, bool INV>
ILS_HD void dft_composite(float2* v) {
  constexpr int R = A * B;
  float2 y[R];
  if constexpr (ct_gcd(A, B) == 1) {
    // Good-Thomas: x[(B n1 + A n2) mod R] -> DFT_A over n1 -> DFT_B over n2 -> X[k], k = k1 (A),
    // k = k2 (B), i.e. k = (k1 B (B^-1 mod A) + k2 A (A^-1 mod B)) mod R
    constexpr int eA = B * ct_modinv(B % A, A), eB = A * ct_modinv(A % B, B);
#pragma unroll
    for (int n2 = 0; n2 < B; ++n2) {
      float2 t[A];
#pragma unroll
      for (int n1 = 0; n1 < A; ++n1) t[n1] = v[(B * n1 + A * n2) % R];
      dft_reg<A, INV>(t);
#pragma unroll
      for (int k1 = 0; k1 < A; ++k1) y[n2 * A + k1] = t[k1];
    }
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) {
      float2 t[B];
#pragma unroll
      for (int n2 = 0; n2 < B; ++n2) t[n2] = y[n2 * A + k1];
      dft_reg<B, INV>(t);
#pragma unroll
      for (int k2 = 0; k2 < B; ++k2) v[(k1 * eA + k2 * eB) % R] = t[k2];
    }
  } else {
    constexpr Roots<R> w{};
#pragma unroll
    for (int n2 = 0; n2 < B; ++n2) {
      float2 t[A];
#pragma unroll
      for (int n1 = 0; n1 < A; ++n1) t[n1] = v[B * n1 + n2];
      dft_reg<A, INV>(t);
#pragma unroll
      for (int k1 = 0; k1 < A; ++k1) y[n2 * A + k1] = twiddle_const<R, INV>(t[k1], n2 * k1, w);
    }
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) {
      float2 t[B];
#pragma unroll
      for (int n2 = 0; n2 < B; ++n2) t[n2] = y[n2 * A + k1];
      dft_reg<B, INV>(t);
#pragma unroll
      for (int k2 = 0; k2 < B; ++k2) v[k1 + A * k2] = t[k2];
    }
  }
}

template <int R, bool INV>
ILS_HD void dft_reg(float2* v) {
  if constexpr (R == 1) {
  } else if constexpr (R == 2) {
    dft2<INV>(v);
  } else if constexpr (R == 3) {
    dft3<INV>(v);
  } else if constexpr (R == 4) {
    dft4<INV>(v);
  } else if constexpr (R == 5) {
    dft5<INV>(v);
  } else if constexpr (R == 8) {
    dft8<INV>(v);
  } else {
    dft_composite<Split<R>::A, Split<R>::B, INV>(v);
  }
}

}  // namespace ils
