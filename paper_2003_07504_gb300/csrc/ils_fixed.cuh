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

// Stage twiddle tables of a plan, r-major so that threads with consecutive k read
// consecutive entries: a stage with stride NS and radix R keeps w_N^{k (N/(NS R)) r} at
// tab[(r - 1) NS + k], r = 1..R-1, k < NS.  Order: forward middle stage (three-stage plans),
// forward last stage, inverse middle stage, inverse last stage (the inverse conjugates).
template <class PL>
struct StageTw {
  static constexpr int N = PL::N, R0 = PL::R0, R1 = PL::R1, RL = PL::RL;
  static constexpr bool MID = PL::STAGES == 3;
  static constexpr int FWD_MID = 0;                                    // NS = R0, R = R1
  static constexpr int FWD_LAST = FWD_MID + (MID ? (R1 - 1) * R0 : 0);   // NS = N / RL, R = RL
  static constexpr int INV_MID = FWD_LAST + (RL - 1) * (N / RL);       // NS = RL, R = R1
  static constexpr int INV_LAST = INV_MID + (MID ? (R1 - 1) * RL : 0);   // NS = N / R0, R = R0
  static constexpr int SIZE = INV_LAST + (R0 - 1) * (N / R0);
};

// bfly with the twiddles of a StageTw table (the same values as root(), read coalesced).
// tab is a global table or a CTA's shared-memory copy (plain loads: either address space).
template <int R, int NS, bool INV>
__device__ __forceinline__ void bfly_tab(float2 (&v)[R], int j, const float2* __restrict__ tab) {
  if constexpr (NS > 1) {
    const int k = j % NS;
#pragma unroll
    for (int r = 1; r < R; ++r) {
      float2 w = tab[(r - 1) * NS + k];
      if (INV) w.y = -w.y;
      v[r] = cmul(v[r], w);
    }
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
