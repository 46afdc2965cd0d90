// Compile-time FFT plans for the common transform lengths.
//
// A FixedPlan<N, R0, R1, R2> is an N-point Stockham FFT (decimation in time) with two
// or three radix stages (R2 == 1 means two).  Stage s with radix R and
// Ns = R0*...*R_{s-1} takes butterfly j (0 <= j < N/R) from inputs j + r N/R,
// twiddles input r by w_N^{(j mod Ns) r N/(Ns R)}, runs the R-point DFT in
// registers and writes output r to (j - j mod Ns) R + (j mod Ns) + r Ns.  The first
// stage (Ns = 1) needs no twiddle and the last stage (Ns = N/R) writes back to the
// positions j + r N/R it read, i.e. outputs land in natural order on the thread
// that read them.  That lets the kernels read the first stage straight from global
// memory, write the last stage straight to global memory, and run "last forward
// stage -> pointwise op -> first inverse stage" without leaving registers.
//
// Threads per sequence: TPS = max_s N / R_s; a thread owns butterfly j = its index
// in every stage where j < N / R_s.
#pragma once
#include <cuda_runtime.h>

#include "ils_dft.cuh"

namespace ils {

__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }

template <int N_, int R0_, int R1_, int R2_ = 1>
struct FixedPlan {
  static constexpr int N = N_;
  static constexpr int R0 = R0_, R1 = R1_, R2 = R2_;
  static constexpr int STAGES = (R2_ == 1) ? 2 : 3;
  static constexpr int RL = (R2_ == 1) ? R1_ : R2_;  // last radix
  static constexpr int TPS = cmax(cmax(N_ / R0_, N_ / R1_), (R2_ == 1) ? 0 : N_ / R2_);
  static_assert(R0_ * R1_ * R2_ == N_, "radices must multiply to N");
};

// w_N^{e} from a table of L-th roots (tw[t] = exp(-2 pi i t / L), L = N * step)
template <bool INV>
__device__ __forceinline__ float2 root(const float2* __restrict__ tw, int e, int step) {
  float2 w = __ldg(&tw[e * step]);
  return INV ? cconj(w) : w;
}

// Twiddle (if Ns > 1) and transform the R inputs of butterfly j.
template <int N, int R, int NS, bool INV>
__device__ __forceinline__ void bfly(float2 (&v)[R], int j, const float2* __restrict__ tw, int step) {
  if constexpr (NS > 1) {
    const int k = j % NS;
    const int e1 = k * (N / (NS * R));
#pragma unroll
    for (int r = 1; r < R; ++r) v[r] = cmul(v[r], root<INV>(tw, e1 * r, step));
  }
  dft_reg<R, INV>(v);
}

// Output position of butterfly j's element r in a stage with radix R and stride NS.
template <int R, int NS>
__device__ __forceinline__ int out_pos(int j, int r) {
  const int k = j % NS;
  return (j - k) * R + k + r * NS;
}

}  // namespace ils
