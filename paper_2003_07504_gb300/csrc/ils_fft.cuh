// Shared-memory mixed-radix FFT building blocks for the ILS kernels (sm_103a).
//
// The FFTs here implement the F and F^-1 of Eq. 9 (Sec. 3.2).  Design:
//  * Stockham autosort, decimation in time, radices 2/3/4/5/8 (every supported
//    length is 2^a 3^b 5^c).  Stage s with radix R and Ns = product of earlier
//    radices maps butterfly j (0 <= j < n/R) from inputs j + r n/R to outputs
//    (j - j%Ns) R + j%Ns + r Ns after twiddling input r by w_n^{(j%Ns) r n/(Ns R)}.
//  * One shared-memory buffer per CTA: each stage gathers every butterfly of
//    the thread into registers, synchronizes, and scatters the results back in
//    place.  A CTA may process several sequences (rows of a strip or columns of
//    a tile) in one sweep.
//  * Twiddles come from a table of L-th roots exp(-2 pi i t / L) computed on
//    the host in double precision (L = the length, or a multiple of it).
//  * Shared-memory indices go through smem_idx(), which inserts one padding
//    element every 16 complex values to spread power-of-two strides over banks.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ils_dft.cuh"

namespace ils {

// A CTA sweeping `elems` complex values with T threads needs elems <= EPT * T,
// where EPT (elements per thread, a template parameter) bounds the registers a
// thread holds during a stage.  Two instantiations exist: 16 (two CTAs per SM)
// and 32 (one CTA per SM, for tiles that do not fit otherwise).
constexpr int kMaxStages = 16;

struct FftPlan {
  int n;                     // transform length
  int nstages;
  int radix[kMaxStages];     // radices in execution order
};

__host__ __device__ __forceinline__ int smem_idx(int i) { return i + (i >> 4); }
__host__ __device__ __forceinline__ int smem_elems(int n) { return n == 0 ? 0 : smem_idx(n - 1) + 1; }

// ---------------------------------------------------------------- one Stockham stage
// Sequences: nseq of length n; element e of sequence s lives at logical index
// s*ss + e*es of `buf` (padded by smem_idx).  tw[t*twstep] = exp(-2 pi i t / n).
// Requires nseq * n <= EPT * blockDim.x.
template <int EPT, int R, bool INV>
__device__ __forceinline__ void stockham_stage(float2* buf, int n, int nseq, int es, int ss, int Ns,
                                               const float2* __restrict__ tw, int twstep) {
  constexpr int B = (EPT + R - 1) / R;
  const int nR = n / R;
  const int total = nseq * nR;
  const int T = blockDim.x;
  const int tws = (n / (Ns * R)) * twstep;
  const int sstride = nR * es;  // source stride between butterfly inputs
  const int dstride = Ns * es;  // destination stride between butterfly outputs
  float2 v[B][R];
  int dbase[B];
#pragma unroll
  for (int b = 0; b < B; ++b) {
    const int w = threadIdx.x + b * T;
    dbase[b] = -1;
    if (w < total) {
      const int s = w / nR;
      const int j = w - s * nR;
      const int k = j % Ns;
      const int sb = s * ss + j * es;
      dbase[b] = s * ss + ((j - k) * R + k) * es;
#pragma unroll
      for (int r = 0; r < R; ++r) v[b][r] = buf[smem_idx(sb + r * sstride)];
      if (Ns > 1) {
        float2 w1 = __ldg(&tw[k * tws]);
        if (INV) w1.y = -w1.y;
        float2 t = w1;
#pragma unroll
        for (int r = 1; r < R; ++r) {
          v[b][r] = cmul(v[b][r], t);
          if (r + 1 < R) t = cmul(t, w1);
        }
      }
      dft_reg<R, INV>(v[b]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < B; ++b) {
    if (dbase[b] >= 0) {
#pragma unroll
      for (int r = 0; r < R; ++r) buf[smem_idx(dbase[b] + r * dstride)] = v[b][r];
    }
  }
  __syncthreads();
}

// Full complex FFT of nseq sequences in place (unnormalized in both directions).
// Callers synchronize before (data in place) - this function synchronizes after.
template <int EPT, bool INV>
__device__ void fft_smem(float2* buf, const FftPlan& plan, int nseq, int es, int ss,
                         const float2* __restrict__ tw, int twstep) {
  int Ns = 1;
  for (int st = 0; st < plan.nstages; ++st) {
    const int R = plan.radix[st];
    switch (R) {
      case 8: stockham_stage<EPT, 8, INV>(buf, plan.n, nseq, es, ss, Ns, tw, twstep); break;
      case 4: stockham_stage<EPT, 4, INV>(buf, plan.n, nseq, es, ss, Ns, tw, twstep); break;
      case 2: stockham_stage<EPT, 2, INV>(buf, plan.n, nseq, es, ss, Ns, tw, twstep); break;
      case 3: stockham_stage<EPT, 3, INV>(buf, plan.n, nseq, es, ss, Ns, tw, twstep); break;
      default: stockham_stage<EPT, 5, INV>(buf, plan.n, nseq, es, ss, Ns, tw, twstep); break;
    }
    Ns *= R;
  }
}

// ---------------------------------------------------------------- real <-> packed half spectrum
// A real row x of even length W = 2M is viewed as M complex z[m] = x[2m] + i x[2m+1].
// After Z = FFT_M(z), the half spectrum X[0..M] of x is
//   X[k] = (Z[k] + conj Z[M-k])/2 - (i/2) w_W^k (Z[k] - conj Z[M-k]),  w_W = exp(-2 pi i/W),
// X[0] and X[M] are real and are packed together as slot 0 = (X[0], X[M]).
// twW[t] = exp(-2 pi i t / W).  Rows: nrows sequences at stride `rs` complex.

__device__ __forceinline__ void r2c_post_pair(float2* buf, int base, int M, int k,
                                              const float2* __restrict__ twW) {
  if (k == 0) {
    float2 z = buf[smem_idx(base)];
    buf[smem_idx(base)] = make_float2(z.x + z.y, z.x - z.y);
    return;
  }
  const int km = M - k;
  const float2 a = buf[smem_idx(base + k)];
  const float2 b = buf[smem_idx(base + km)];
  // X[k]
  {
    const float2 cb = cconj(b);
    const float2 fe = cscale(cadd(a, cb), 0.5f);
    const float2 fo = cscale(csub(a, cb), 0.5f);      // times -i below
    const float2 w = __ldg(&twW[k]);
    const float2 x = cadd(fe, cmul(w, make_float2(fo.y, -fo.x)));
    buf[smem_idx(base + k)] = x;
  }
  if (km != k) {
    const float2 ca = cconj(a);
    const float2 fe = cscale(cadd(b, ca), 0.5f);
    const float2 fo = cscale(csub(b, ca), 0.5f);
    const float2 w = __ldg(&twW[km]);
    const float2 x = cadd(fe, cmul(w, make_float2(fo.y, -fo.x)));
    buf[smem_idx(base + km)] = x;
  }
}

// Inverse of the packing above, unnormalized: produces Z with IFFT_M(Z) = W * z.
__device__ __forceinline__ void c2r_pre_pair(float2* buf, int base, int M, int k,
                                             const float2* __restrict__ twW) {
  if (k == 0) {
    float2 x = buf[smem_idx(base)];
    buf[smem_idx(base)] = make_float2(x.x + x.y, x.x - x.y);
    return;
  }
  const int km = M - k;
  const float2 a = buf[smem_idx(base + k)];
  const float2 b = buf[smem_idx(base + km)];
  {
    const float2 cb = cconj(b);
    const float2 s = cadd(a, cb);
    const float2 d = csub(a, cb);
    const float2 w = cconj(__ldg(&twW[k]));            // exp(+2 pi i k / W)
    const float2 t = cmul(w, d);
    buf[smem_idx(base + k)] = make_float2(s.x - t.y, s.y + t.x);   // s + i t
  }
  if (km != k) {
    const float2 ca = cconj(a);
    const float2 s = cadd(b, ca);
    const float2 d = csub(b, ca);
    const float2 w = cconj(__ldg(&twW[km]));
    const float2 t = cmul(w, d);
    buf[smem_idx(base + km)] = make_float2(s.x - t.y, s.y + t.x);
  }
}

}  // namespace ils
