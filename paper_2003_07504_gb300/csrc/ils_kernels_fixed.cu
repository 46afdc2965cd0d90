// ILS kernels specialised at compile time for the common transform lengths (the
// 1920x1080 and 3840x2160 frames, the 256x256 parity image and the batch sizes).
// Same passes and spectrum layout as the generic kernels in ils_kernels.cu (see the
// description there); what changes is how each FFT runs:
//  * radix plans of two or three stages with composite radices up to 16 held in
//    registers (ils_fixed.cuh), so an FFT costs one or two shared-memory exchanges;
//  * the first stage reads global memory directly and the last stage writes it
//    directly (the c2r/r2c packing is folded into those reads/writes);
//  * the column pass runs last-forward-stage -> Eq. 9 division -> first-inverse-stage
//    in registers;
//  * one tile (a strip of rows or a group of columns) per CTA.  (A persistent
//    grid-stride loop over tiles made the compiler hoist every per-thread shared-memory
//    address and twiddle out of the loop, which spilled registers.)
#include <cuda_runtime.h>

#include "ils_fixed.cuh"
#include "ils_internal.h"

namespace ils {
namespace {

__device__ __forceinline__ int wrap_row(int y, int H) { return y < 0 ? y + H : (y >= H ? y - H : y); }

// Shared memory of a column-pass CTA: the tile of G columns, padded by smem_idx.  (Copying the
// plan's stage-twiddle table and the y denominator into shared memory as well measured 4 %
// slower at 1080 rows: those reads hit L1 and are shared by the tile's columns.)
template <class PL, int G>
constexpr size_t col_smem_bytes() {  // smem_elems(N G) complex (one padding slot per 16)
  return (size_t)(PL::N * G + (PL::N * G - 1) / 16) * sizeof(float2);
}

// In place on nrows smem rows of packed half spectra X (slot 0 = (X[0], X[M])): replace X
// by Z, the half-length sequence whose unnormalized inverse FFT is W (x[2m] + i x[2m+1]):
// Z[k] = (X[k] + conj X[M-k]) + i e^{+2 pi i k/W} (X[k] - conj X[M-k]);  Z[0] = (X0+XM, X0-XM).
// Thread-strided over the pairs (k, M-k); the caller synchronizes before and after.
template <int M>
__device__ __forceinline__ void unpack_c2r_rows(float2* sm, int nrows, const float2* __restrict__ twW) {
  constexpr int P = M / 2 + 1;
  for (int w = threadIdx.x; w < nrows * P; w += blockDim.x) {
    const int r = w / P;
    const int k = w - r * P;
    const int b = r * M;
    if (k == 0) {
      const float2 x = sm[smem_idx(b)];
      sm[smem_idx(b)] = c2(x.x + x.y, x.x - x.y);
      continue;
    }
    const float2 a = sm[smem_idx(b + k)], bb = sm[smem_idx(b + M - k)];
    {
      const float2 cb = cconj(bb);
      const float2 sum = cadd(a, cb), d = csub(a, cb);
      const float2 tt = cmul(cconj(__ldg(&twW[k])), d);
      sm[smem_idx(b + k)] = c2(sum.x - tt.y, sum.y + tt.x);
    }
    if (M - k != k) {
      const float2 ca = cconj(a);
      const float2 sum = cadd(bb, ca), d = csub(bb, ca);
      const float2 tt = cmul(cconj(__ldg(&twW[M - k])), d);
      sm[smem_idx(b + M - k)] = c2(sum.x - tt.y, sum.y + tt.x);
    }
  }
}

// X[k] of a real row from Z = FFT_M(x[2m] + i x[2m+1]): a = Z[k], b = Z[M-k].
__device__ __forceinline__ float2 r2c_x(float2 a, float2 b, int k, const float2* __restrict__ twW) {
  const float2 cb = cconj(b);
  const float2 fe = cscale(cadd(a, cb), 0.5f);
  const float2 fo = cscale(csub(a, cb), 0.5f);
  return cadd(fe, cmul(__ldg(&twW[k]), c2(fo.y, -fo.x)));
}

// ---------------------------------------------------------------- column pass
template <class PL, int G, int MINB>
__global__ void __launch_bounds__(G * PL::TPS, MINB)
col_fixed_kernel(int M, int C, const float2* __restrict__ twc, const float* __restrict__ ax,
                 const float* __restrict__ by, float scale, float2* __restrict__ spec) {
  griddep_launch();
  griddep_wait();
  constexpr int N = PL::N, R0 = PL::R0, R1 = PL::R1, RL = PL::RL;
  constexpr int NS0 = N / R0, NS1 = N / R1, NSL = N / RL;
  using TW = StageTw<PL>;  // twc: this plan's stage twiddle tables
  extern __shared__ float2 sm[];
  const int tiles_per_ch = (M + G - 1) / G;
  const int ntiles = tiles_per_ch * C;
  {
    const int tile = blockIdx.x;
    if (tile >= ntiles) return;
    const int t = (int)threadIdx.x, g = t % G, j = t / G;
    auto S = [&](int l) -> float2& { return sm[smem_idx(l * G + g)]; };
    const int ch = tile / tiles_per_ch;
    const int k0 = (tile - ch * tiles_per_ch) * G;
    const int k = k0 + g;
    const bool live = k < M;
    float2* col = spec + (size_t)ch * N * M + (live ? k : 0);
    // coalesced copy of the tile (G complex per row) into smem with every load of a thread
    // in flight at once (compile-time trip count), then forward stage 0 (Ns = 1)
    {
      const float2* tilep = spec + (size_t)ch * N * M + k0;
      constexpr int T = G * PL::TPS, PER = (N * G + T - 1) / T, BATCH = PER < 24 ? PER : 24;
#pragma unroll
      for (int q0 = 0; q0 < PER; q0 += BATCH) {
        float2 ld[BATCH];
#pragma unroll
        for (int q = 0; q < BATCH; ++q) {
          const int w = t + (q0 + q) * T;
          const int l = w / G, gg = w - (w / G) * G;
          ld[q] = (q0 + q < PER && w < N * G && k0 + gg < M) ? tilep[(size_t)l * M + gg] : c2(0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < BATCH; ++q)
          if (q0 + q < PER && t + (q0 + q) * T < N * G) sm[smem_idx(t + (q0 + q) * T)] = ld[q];
      }
      __syncthreads();
      float2 v[R0];
      if (j < NS0) {
#pragma unroll
        for (int r = 0; r < R0; ++r) v[r] = S(j + r * NS0);
        dft_reg<R0, false>(v);
      }
      __syncthreads();
      if (j < NS0) {
#pragma unroll
        for (int r = 0; r < R0; ++r) S(j * R0 + r) = v[r];
      }
      __syncthreads();
    }
    if constexpr (PL::STAGES == 3) {
      float2 v[R1];
      if (j < NS1) {
#pragma unroll
        for (int r = 0; r < R1; ++r) v[r] = S(j + r * NS1);
        bfly_tab<R1, R0, false>(v, j, twc + TW::FWD_MID);
      }
      __syncthreads();
      if (j < NS1) {
#pragma unroll
        for (int r = 0; r < R1; ++r) S(out_pos<R1, R0>(j, r)) = v[r];
      }
      __syncthreads();
    }
    // last forward stage -> divide by the Eq. 9 denominator (and 1/(HW)) -> first inverse stage
    {
      float2 v[RL];
      if (j < NSL) {
#pragma unroll
        for (int r = 0; r < RL; ++r) v[r] = S(j + r * NSL);
        bfly_tab<RL, NSL, false>(v, j, twc + TW::FWD_LAST);
      }
      if (k0 == 0) {
        // Column 0 packs two real columns: Z = A + iB with A = F(X[:,0]), B = F(X[:,M]).
        // A/dA + iB/dB = Z[l] (1/dA + 1/dB)/2 + conj(Z[N-l]) (1/dA - 1/dB)/2.
        __syncthreads();
        if (j < NSL) {
#pragma unroll
          for (int r = 0; r < RL; ++r) S(j + r * NSL) = v[r];
        }
        __syncthreads();
        if (g == 0 && j < NSL) {
          const float axM = __ldg(&ax[M]);
#pragma unroll
          for (int r = 0; r < RL; ++r) {
            const int l = j + r * NSL;
            const float2 zm = S(l == 0 ? 0 : N - l);
            const float byl = __ldg(&by[l]);
            const float ia = __fdividef(1.0f, 1.0f + byl);
            const float ib = __fdividef(1.0f, 1.0f + axM + byl);
            const float sp = 0.5f * scale * (ia + ib), sn = 0.5f * scale * (ia - ib);
            v[r] = c2(sp * v[r].x + sn * zm.x, sp * v[r].y - sn * zm.y);
          }
        }
      }
      if (j < NSL && !(k0 == 0 && g == 0)) {
        const float axk = __ldg(&ax[live ? k : 0]);
#pragma unroll
        for (int r = 0; r < RL; ++r) {
          const float s = __fdividef(scale, 1.0f + axk + __ldg(&by[j + r * NSL]));
          v[r] = cscale(v[r], s);
        }
      }
      if (j < NSL) dft_reg<RL, true>(v);
      __syncthreads();
      if (j < NSL) {
#pragma unroll
        for (int r = 0; r < RL; ++r) S(j * RL + r) = v[r];
      }
      __syncthreads();
    }
    if constexpr (PL::STAGES == 3) {
      float2 v[R1];
      if (j < NS1) {
#pragma unroll
        for (int r = 0; r < R1; ++r) v[r] = S(j + r * NS1);
        bfly_tab<R1, RL, true>(v, j, twc + TW::INV_MID);
      }
      __syncthreads();
      if (j < NS1) {
#pragma unroll
        for (int r = 0; r < R1; ++r) S(out_pos<R1, RL>(j, r)) = v[r];
      }
      __syncthreads();
    }
    // last inverse stage (radix R0, Ns = N/R0) straight to global memory
    {
      float2 v[R0];
      if (j < NS0) {
#pragma unroll
        for (int r = 0; r < R0; ++r) v[r] = S(j + r * NS0);
        bfly_tab<R0, NS0, true>(v, j, twc + TW::INV_LAST);
        if (live) {
#pragma unroll
          for (int r = 0; r < R0; ++r) col[(size_t)(j + r * NS0) * M] = v[r];
        }
      }
    }
  }
}

// ---------------------------------------------------------------- row passes
// Inverse real row FFT of row `i` of the strip (global spectrum row X) into smem row i,
// natural order (complex m holds pixels 2m, 2m+1).  All threads call it (syncs inside).
template <class PL, int EPI = 0>
__device__ __forceinline__ void fft_rows_smem_inverse(float2* sm, int i, int j, bool live,
                                                      const float2* __restrict__ twr, float2* out, size_t rowoff,
                                                      const Epilogue* epi);

// Inverse real row FFT of strip rows 0..nrows-1 (global spectrum rows X(i)) into smem rows
// 0..nrows-1 in natural order (complex m holds pixels 2m, 2m+1).  Three barrier-separated
// phases keep the register footprint of each small: a coalesced copy of the packed rows,
// the c2r un-packing of pairs (k, M-k) in place, then the FFT stages.  All threads call it.
template <class PL, class RowPtr>
__device__ __forceinline__ void rows_inverse_to_smem(float2* sm, int nrows, int i, int j, RowPtr X,
                                                     const float2* __restrict__ twW, const float2* __restrict__ twr) {
  constexpr int M = PL::N;
  const int t = threadIdx.x, T = blockDim.x;
  __syncthreads();  // the previous user of the buffer is done
  for (int w = t; w < nrows * M; w += T) {
    const int r = w / M;
    const int m = w - r * M;
    sm[smem_idx(w)] = X(r)[m];
  }
  __syncthreads();
  unpack_c2r_rows<M>(sm, nrows, twW);
  __syncthreads();
  fft_rows_smem_inverse<PL>(sm, i, j, i < nrows, twr, nullptr, 0, nullptr);
}

// The inverse FFT stages on smem row i (input natural order, output natural order, to
// smem row i, or, when out is not null, to pixel pairs rowoff + m of the global output
// image through the epilogue).  twr: the plan's StageTw table (forward-stage parts: the
// inverse runs the stages in the forward order and conjugates).
template <class PL, int EPI>
__device__ __forceinline__ void fft_rows_smem_inverse(float2* sm, int i, int j, bool live,
                                                      const float2* __restrict__ twr, float2* out, size_t rowoff,
                                                      const Epilogue* epi) {
  using TW = StageTw<PL>;
  constexpr int M = PL::N, R0 = PL::R0, R1 = PL::R1, RL = PL::RL;
  constexpr int NS0 = M / R0, NS1 = M / R1, NSL = M / RL;
  auto U = [&](int m) -> float2& { return sm[smem_idx(i * M + m)]; };
  {
    float2 v[R0];
    if (live && j < NS0) {
#pragma unroll
      for (int r = 0; r < R0; ++r) v[r] = U(j + r * NS0);
      dft_reg<R0, true>(v);
    }
    __syncthreads();
    if (live && j < NS0) {
#pragma unroll
      for (int r = 0; r < R0; ++r) U(j * R0 + r) = v[r];
    }
    __syncthreads();
  }
  if constexpr (PL::STAGES == 3) {
    float2 v[R1];
    if (live && j < NS1) {
#pragma unroll
      for (int r = 0; r < R1; ++r) v[r] = U(j + r * NS1);
      bfly_tab<R1, R0, true>(v, j, twr + TW::FWD_MID);
    }
    __syncthreads();
    if (live && j < NS1) {
#pragma unroll
      for (int r = 0; r < R1; ++r) U(out_pos<R1, R0>(j, r)) = v[r];
    }
    __syncthreads();
  }
  {
    float2 v[RL];
    if (live && j < NSL) {
#pragma unroll
      for (int r = 0; r < RL; ++r) v[r] = U(j + r * NSL);
      bfly_tab<RL, NSL, true>(v, j, twr + TW::FWD_LAST);
    }
    if (out != nullptr) {
      float dm = 0.0f;
      if (live && j < NSL) {
#pragma unroll
        for (int r = 0; r < RL; ++r) dm = fmaxf(dm, epi->template store<EPI>(out, rowoff + j + r * NSL, v[r]));
      }
      epi->template finish<EPI>(dm);
      return;
    }
    __syncthreads();
    if (live && j < NSL) {
#pragma unroll
      for (int r = 0; r < RL; ++r) U(j + r * NSL) = v[r];
    }
    __syncthreads();
  }
}

// Fused row pass of one iteration: grid-stride over strips of ROWS rows (all channels);
// CTA = (ROWS + 2) x TPS threads.  In the inverse FFT thread (i, j) works on strip row i
// (i = 0 and ROWS+1 are the halo rows y0-1 and y0+ROWS); the stencil runs over all
// threads row by row; the forward FFT of output row o runs on threads (o, j).
template <class PL, int ROWS, bool FIRST, int PEN>
__global__ void __launch_bounds__((ROWS + 2) * PL::TPS, 1)
row_fwd_fixed_kernel(int H, int C, const float2* __restrict__ twW, const float2* __restrict__ twr, MuParams mp,
                     const float* __restrict__ f, const float* __restrict__ u0, const float2* __restrict__ spec_in,
                     float2* __restrict__ spec_out, float* __restrict__ u_ckpt) {
  griddep_launch();
  griddep_wait();
  using TW = StageTw<PL>;  // twr: this plan's stage twiddle tables
  constexpr int M = PL::N, R0 = PL::R0, R1 = PL::R1, RL = PL::RL, TPS = PL::TPS;
  constexpr int NS0 = M / R0, NS1 = M / R1, NSL = M / RL;
  constexpr int P = M / 2 + 1;
  extern __shared__ float2 sm[];
  const int strips = (H + ROWS - 1) / ROWS;
  const size_t plane = (size_t)H * M;
  auto U = [&](int row, int m) -> float2& { return sm[smem_idx(row * M + m)]; };
  {
    const int tile = blockIdx.x;
    if (tile >= strips * C) return;
    const int t = (int)threadIdx.x, i = t / TPS, j = t - (t / TPS) * TPS;
    const int ch = tile / strips;
    const int y0 = (tile - ch * strips) * ROWS;
    const int nout = min(ROWS, H - y0);
    // (a) u^n on strip rows 0 .. nout+1 into shared memory
    if (FIRST) {
      const float2* src = reinterpret_cast<const float2*>(u0 != nullptr ? u0 : f) + ch * plane;
      __syncthreads();
      for (int w = t; w < (nout + 2) * M; w += blockDim.x) {
        const int r = w / M;
        const int m = w - r * M;
        sm[smem_idx(w)] = src[(size_t)wrap_row(y0 - 1 + r, H) * M + m];
      }
      __syncthreads();
    } else {
      const float2* base = spec_in + ch * plane;
      auto X = [&](int r) { return base + (size_t)wrap_row(y0 - 1 + r, H) * M; };
      rows_inverse_to_smem<PL>(sm, nout + 2, i, j, X, twW, twr);
    }
    // (b) r = f + lambda/2 (grad_x^T mu_x + grad_y^T mu_y), one output row at a time.  Row o
    // (strip row o+1) reads u rows o, o+1, o+2 and is then written into slot o, whose u row no
    // later output row needs; one barrier per row separates the reads from the write.
    {
      constexpr int IPT = (M + (ROWS + 2) * TPS - 1) / ((ROWS + 2) * TPS);  // items per thread per row
      const int T = blockDim.x;
      for (int o = 0; o < nout; ++o) {
        const size_t rowoff = ch * plane + (size_t)(y0 + o) * M;
        const float2* fr = reinterpret_cast<const float2*>(f) + rowoff;
        float2 rv[IPT];
#pragma unroll
        for (int q = 0; q < IPT; ++q) {
          const int m = t + q * T;
          if (m < M && mp.half_lambda == 0.0f) {   // lambda = 0 (or a plain row FFT): r = f
            rv[q] = fr[m];
            if (u_ckpt != nullptr) reinterpret_cast<float2*>(u_ckpt)[rowoff + m] = U(o + 1, m);
          } else if (m < M) {
            const float2 c = U(o + 1, m);
            const float ul = U(o + 1, m == 0 ? M - 1 : m - 1).y;
            const float ur = U(o + 1, m == M - 1 ? 0 : m + 1).x;
            const float2 up = U(o, m);
            const float2 dn = U(o + 2, m);
            const float2 fv = fr[m];
            const float mx_l = mu_pen<PEN>(c.x - ul, mp);
            const float mx_c = mu_pen<PEN>(c.y - c.x, mp);
            const float mx_r = mu_pen<PEN>(ur - c.y, mp);
            const float my0u = mu_pen<PEN>(c.x - up.x, mp);
            const float my0d = mu_pen<PEN>(dn.x - c.x, mp);
            const float my1u = mu_pen<PEN>(c.y - up.y, mp);
            const float my1d = mu_pen<PEN>(dn.y - c.y, mp);
            rv[q] = c2(fmaf(mp.half_lambda, (mx_l - mx_c) + (my0u - my0d), fv.x),
                       fmaf(mp.half_lambda, (mx_c - mx_r) + (my1u - my1d), fv.y));
            if (u_ckpt != nullptr) reinterpret_cast<float2*>(u_ckpt)[rowoff + m] = c;
          }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < IPT; ++q) {
          const int m = t + q * T;
          if (m < M) U(o, m) = rv[q];
        }
      }
      __syncthreads();
    }
    // forward row FFT of r rows (slots 0 .. nout-1)
    const bool outlive = i < nout;
    {
      float2 v[R0];
      if (outlive && j < NS0) {
#pragma unroll
        for (int r = 0; r < R0; ++r) v[r] = U(i, j + r * NS0);
        dft_reg<R0, false>(v);
      }
      __syncthreads();
      if (outlive && j < NS0) {
#pragma unroll
        for (int r = 0; r < R0; ++r) U(i, j * R0 + r) = v[r];
      }
      __syncthreads();
    }
    if constexpr (PL::STAGES == 3) {
      float2 v[R1];
      if (outlive && j < NS1) {
#pragma unroll
        for (int r = 0; r < R1; ++r) v[r] = U(i, j + r * NS1);
        bfly_tab<R1, R0, false>(v, j, twr + TW::FWD_MID);
      }
      __syncthreads();
      if (outlive && j < NS1) {
#pragma unroll
        for (int r = 0; r < R1; ++r) U(i, out_pos<R1, R0>(j, r)) = v[r];
      }
      __syncthreads();
    }
    {
      float2 v[RL];
      if (outlive && j < NSL) {
#pragma unroll
        for (int r = 0; r < RL; ++r) v[r] = U(i, j + r * NSL);
        bfly_tab<RL, NSL, false>(v, j, twr + TW::FWD_LAST);
      }
      __syncthreads();
      if (outlive && j < NSL) {
#pragma unroll
        for (int r = 0; r < RL; ++r) U(i, j + r * NSL) = v[r];
      }
      __syncthreads();
    }
    // (c) real-row packing and store: slots 0..nout-1, pairs (k, M-k)
    for (int w = t; w < nout * P; w += blockDim.x) {
      const int o = w / P;
      const int k = w - o * P;
      float2* dst = spec_out + ch * plane + (size_t)(y0 + o) * M;
      if (k == 0) {
        const float2 z = U(o, 0);
        dst[0] = c2(z.x + z.y, z.x - z.y);
      } else {
        const float2 a = U(o, k), b = U(o, M - k);
        dst[k] = r2c_x(a, b, k, twW);
        if (M - k != k) dst[M - k] = r2c_x(b, a, M - k, twW);
      }
    }
  }
}

// Final inverse row pass: strips of ROWS rows, last stage written straight to u.
template <class PL, int ROWS, int EPI>
__global__ void __launch_bounds__(ROWS * PL::TPS, 1)
row_inv_fixed_kernel(int H, int C, const float2* __restrict__ twW, const float2* __restrict__ twr,
                     const float2* __restrict__ spec, float* __restrict__ u, Epilogue epi) {
  griddep_launch();
  griddep_wait();
  constexpr int M = PL::N, TPS = PL::TPS;
  extern __shared__ float2 sm[];
  const int strips = (H + ROWS - 1) / ROWS;
  const size_t plane = (size_t)H * M;
  {
    const int tile = blockIdx.x;
    if (tile >= strips * C) return;
    const int t = (int)threadIdx.x, i = t / TPS, j = t - (t / TPS) * TPS;
    const int ch = tile / strips;
    const int y0 = (tile - ch * strips) * ROWS;
    const int n = min(ROWS, H - y0);
    const float2* base = spec + ch * plane + (size_t)y0 * M;
    // the phases of rows_inverse_to_smem, with the last stage stored to u
    __syncthreads();
    for (int w = t; w < n * M; w += blockDim.x) sm[smem_idx(w)] = base[w];
    __syncthreads();
    unpack_c2r_rows<M>(sm, n, twW);
    __syncthreads();
    const size_t rowoff = ch * plane + (size_t)(y0 + (i < n ? i : 0)) * M;
    fft_rows_smem_inverse<PL, EPI>(sm, i, j, i < n, twr, reinterpret_cast<float2*>(u), rowoff, &epi);
  }
}

// ---------------------------------------------------------------- registry

using RowFwdFn = void (*)(int, int, const float2*, const float2*, MuParams, const float*, const float*, const float2*,
                          float2*, float*);
using RowInvFn = void (*)(int, int, const float2*, const float2*, const float2*, float*, Epilogue);
using ColFn = void (*)(int, int, const float2*, const float*, const float*, float, float2*);

struct RowEntry {
  int M, tps, rows_fwd, rows_inv;
  RowFwdFn first[kPenalties], later[kPenalties];  // per penalty (MuParams::pen)
  RowInvFn inv[kEpilogues];     // per epilogue mode
  int R0, R1, R2, tw;           // radices (R2 = 1: two stages) and StageTw size
};
struct ColEntry {
  int H, tps, G;
  ColFn fn;
  int R0, R1, R2, tw;  // radices (R2 = 1: two stages) and StageTw size
  size_t smem;         // dynamic shared memory per CTA (col_smem_bytes)
};

template <class PL, int RF, int RI>
constexpr RowEntry row_entry() {
  static_assert((RF + 2) * PL::TPS <= 1024 && RI * PL::TPS <= 1024, "at most 1024 threads per CTA");
  return RowEntry{PL::N,
                  PL::TPS,
                  RF,
                  RI,
                  {row_fwd_fixed_kernel<PL, RF, true, 0>, row_fwd_fixed_kernel<PL, RF, true, 1>,
                   row_fwd_fixed_kernel<PL, RF, true, 2>},
                  {row_fwd_fixed_kernel<PL, RF, false, 0>, row_fwd_fixed_kernel<PL, RF, false, 1>,
                   row_fwd_fixed_kernel<PL, RF, false, 2>},
                  {row_inv_fixed_kernel<PL, RI, 0>, row_inv_fixed_kernel<PL, RI, 1>, row_inv_fixed_kernel<PL, RI, 2>,
                   row_inv_fixed_kernel<PL, RI, 3>, row_inv_fixed_kernel<PL, RI, 4>, row_inv_fixed_kernel<PL, RI, 5>},
                  PL::R0, PL::R1, PL::R2, StageTw<PL>::SIZE};
}
template <class PL, int G, int MINB = 1>
constexpr ColEntry col_entry() {
  return ColEntry{PL::N,  PL::TPS, G, col_fixed_kernel<PL, G, MINB>, PL::R0, PL::R1, PL::R2, StageTw<PL>::SIZE,
                  col_smem_bytes<PL, G>()};
}

// Several entries may share a length: the first is the default, the others are
// alternative tile shapes the batch autotuner may pick.
const RowEntry kRows[] = {
    row_entry<FixedPlan<128, 8, 16>, 8, 8>(),
    row_entry<FixedPlan<320, 8, 8, 5>, 6, 8>(),
    row_entry<FixedPlan<640, 8, 8, 10>, 6, 8>(),
    row_entry<FixedPlan<960, 10, 12, 8>, 6, 8>(),
    row_entry<FixedPlan<1024, 8, 8, 16>, 4, 6>(),
    row_entry<FixedPlan<1920, 16, 12, 10>, 3, 4>(),
    row_entry<FixedPlan<960, 10, 12, 8>, 2, 4>(),
    row_entry<FixedPlan<640, 8, 8, 10>, 2, 4>(),
};
// Defaults are the fastest shapes measured by the batch autotuner on GB300 at
// 640x480, 1280x720, 1920x1080, 2048x1536 and 3840x2160 RGB.  One default per length, whatever
// the channel count, so that a channel's result does not depend on the other channels of
// the call (at 1080 rows: 36 x 30 with 8 columns per CTA, 1920 x 1080 RGB 265 us per frame
// against 270 for 12 x 10 x 9 and 272-276 for 4 columns per CTA; gray 178 against 173 / 176;
// at 2160 rows: 45 x 48 with 8 columns per CTA, one CTA per SM at 168 registers, 3840 x 2160
// RGB column pass 106 us per launch and 1078 us per N = 4 frame against 112 / 1156 us with 4
// columns at two CTAs per SM and 139 / 1219 us with 6 columns at one).
const ColEntry kCols[] = {
    col_entry<FixedPlan<256, 16, 16>, 16>(),
    col_entry<FixedPlan<480, 8, 6, 10>, 4, 2>(),
    col_entry<FixedPlan<720, 8, 9, 10>, 4, 2>(),
    col_entry<FixedPlan<1080, 36, 30>, 8, 2>(),
    col_entry<FixedPlan<1536, 32, 48>, 4, 2>(),
    col_entry<FixedPlan<2160, 45, 48>, 8>(),
    col_entry<FixedPlan<512, 16, 32>, 4, 3>(),
    // alternatives for the autotuner
    col_entry<FixedPlan<1080, 12, 10, 9>, 4, 2>(),
    col_entry<FixedPlan<1080, 36, 30>, 4, 3>(),
    col_entry<FixedPlan<1080, 30, 36>, 8>(),
    col_entry<FixedPlan<1080, 36, 30>, 6, 3>(),
    col_entry<FixedPlan<1080, 36, 30>, 4, 4>(),
    col_entry<FixedPlan<720, 24, 30>, 4, 3>(),
    col_entry<FixedPlan<480, 20, 24>, 4, 4>(),
    col_entry<FixedPlan<1536, 16, 12, 8>, 4>(),
    col_entry<FixedPlan<2160, 12, 12, 15>, 4>(),
    col_entry<FixedPlan<512, 8, 8, 8>, 4, 2>(),
    col_entry<FixedPlan<2160, 45, 48>, 4, 2>(),
    col_entry<FixedPlan<1536, 32, 48>, 8>(),
    col_entry<FixedPlan<720, 24, 30>, 8, 2>(),
    col_entry<FixedPlan<480, 20, 24>, 8, 2>(),
};

}  // namespace

// ---------------------------------------------------------------- host interface

int fixed_row_index(int M) {
  for (int i = 0; i < (int)(sizeof(kRows) / sizeof(kRows[0])); ++i)
    if (kRows[i].M == M) return i;
  return -1;
}
int fixed_col_index(int H) {
  for (int i = 0; i < (int)(sizeof(kCols) / sizeof(kCols[0])); ++i)
    if (kCols[i].H == H) return i;
  return -1;
}

int fixed_row_variants(int M, int* idx, int max) {
  int n = 0;
  for (int i = 0; i < (int)(sizeof(kRows) / sizeof(kRows[0])) && n < max; ++i)
    if (kRows[i].M == M) idx[n++] = i;
  return n;
}
int fixed_col_variants(int H, int* idx, int max) {
  int n = 0;
  for (int i = 0; i < (int)(sizeof(kCols) / sizeof(kCols[0])) && n < max; ++i)
    if (kCols[i].H == H) idx[n++] = i;
  return n;
}

// Twiddle entries of a column table (Tables::twH) for length H: the H roots, then the
// StageTw tables of every compile-time plan of H in kCols order.
size_t col_twiddle_count(int H) {
  size_t n = H;
  for (const ColEntry& c : kCols)
    if (c.H == H) n += c.tw;
  return n;
}

// Entries of a row table (Tables::twW) for row length W: the W roots, the M = W/2 four-step
// entries of the warp-per-row kernels, then the StageTw tables of every compile-time row plan
// of M in kRows order.
size_t row_twiddle_count(int W) {
  size_t n = (size_t)W + W / 2;
  for (const RowEntry& r : kRows)
    if (r.M == W / 2) n += r.tw;
  return n;
}

namespace {
size_t row_tw_offset(int idx) {
  size_t off = (size_t)3 * kRows[idx].M;
  for (int i = 0; i < idx; ++i)
    if (kRows[i].M == kRows[idx].M) off += kRows[i].tw;
  return off;
}

size_t col_tw_offset(int idx) {
  size_t off = kCols[idx].H;
  for (int i = 0; i < idx; ++i)
    if (kCols[i].H == kCols[idx].H) off += kCols[i].tw;
  return off;
}

// One StageTw table gathered from the roots: stage (R, NS) entries
// tab[(r - 1) NS + k] = tw[step k (N / (NS R)) r] (tw holds the (step N)-th roots of unity).
__global__ void stage_tw_kernel(int N, int R0, int R1, int R2, int step, const float2* __restrict__ tw,
                                float2* __restrict__ tab) {
  const bool mid = R2 > 1;
  const int RL = mid ? R2 : R1;
  // (NS, R) of the four stage tables in StageTw order; zero-size where absent
  const int ns[4] = {R0, N / RL, RL, N / R0};
  const int rr[4] = {mid ? R1 : 1, RL, mid ? R1 : 1, R0};
  int base = 0;
  for (int s = 0; s < 4; ++s) {
    const int n = (rr[s] - 1) * ns[s];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      const int r = 1 + i / ns[s], k = i % ns[s];
      tab[base + i] = tw[step * k * (N / (ns[s] * rr[s])) * r];
    }
    base += n;
  }
}
}  // namespace

cudaError_t build_col_twiddles(int H, float2* twH, cudaStream_t st) {
  for (int i = 0; i < (int)(sizeof(kCols) / sizeof(kCols[0])); ++i) {
    const ColEntry& c = kCols[i];
    if (c.H != H) continue;
    stage_tw_kernel<<<(c.tw + 255) / 256, 256, 0, st>>>(c.H, c.R0, c.R1, c.R2, 1, twH, twH + col_tw_offset(i));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t build_row_twiddles(int W, float2* twW, cudaStream_t st) {
  for (int i = 0; i < (int)(sizeof(kRows) / sizeof(kRows[0])); ++i) {
    const RowEntry& r = kRows[i];
    if (r.M != W / 2) continue;
    stage_tw_kernel<<<(r.tw + 255) / 256, 256, 0, st>>>(r.M, r.R0, r.R1, r.R2, 2, twW, twW + row_tw_offset(i));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static size_t row_smem(int rows, int M) { return (size_t)smem_elems(rows * M) * sizeof(float2); }

cudaError_t fixed_set_attributes() {
  cudaError_t e;
  for (const RowEntry& r : kRows) {
    const int sf = (int)row_smem(r.rows_fwd + 2, r.M), si = (int)row_smem(r.rows_inv, r.M);
    for (int pen = 0; pen < kPenalties; ++pen) {
      if ((e = cudaFuncSetAttribute(r.first[pen], cudaFuncAttributeMaxDynamicSharedMemorySize, sf))) return e;
      if ((e = cudaFuncSetAttribute(r.later[pen], cudaFuncAttributeMaxDynamicSharedMemorySize, sf))) return e;
    }
    for (int m = 0; m < kEpilogues; ++m)
      if ((e = cudaFuncSetAttribute(r.inv[m], cudaFuncAttributeMaxDynamicSharedMemorySize, si))) return e;
  }
  for (const ColEntry& c : kCols) {
    const int s = (int)c.smem;
    if ((e = cudaFuncSetAttribute(c.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, s))) return e;
  }
  return cudaSuccess;
}

cudaError_t fixed_row_forward(int idx, const ImageDesc& d, const Tables& t, const MuParams& mp, const float* f,
                              const float* u0, const float2* spec_in, float2* spec_out, float* u_ckpt,
                              cudaStream_t stream) {
  const RowEntry& r = kRows[idx];
  const int threads = (r.rows_fwd + 2) * r.tps;
  const size_t smem = row_smem(r.rows_fwd + 2, r.M);
  const int tiles = (d.H + r.rows_fwd - 1) / r.rows_fwd * d.C;
  const int pen = mp.pen;
  RowFwdFn fn = spec_in == nullptr ? r.first[pen] : r.later[pen];
  return launch_k(d.pdl, fn, tiles, threads, smem, stream, d.H, d.C, t.twW, t.twW + row_tw_offset(idx), mp, f, u0,
                  spec_in, spec_out, u_ckpt);
}

cudaError_t fixed_row_inverse(int idx, const ImageDesc& d, const Tables& t, const float2* spec, float* u,
                              cudaStream_t stream, const Epilogue& epi) {
  const RowEntry& r = kRows[idx];
  const int threads = r.rows_inv * r.tps;
  const size_t smem = row_smem(r.rows_inv, r.M);
  const int tiles = (d.H + r.rows_inv - 1) / r.rows_inv * d.C;
  return launch_k(d.pdl, r.inv[epi.mode], tiles, threads, smem, stream, d.H, d.C, t.twW, t.twW + row_tw_offset(idx),
                  spec, u, epi);
}

cudaError_t fixed_col_solve(int idx, const ImageDesc& d, const Tables& t, float2* spec, cudaStream_t stream) {
  const ColEntry& c = kCols[idx];
  const int M = d.W / 2;
  const int threads = c.G * c.tps;
  const size_t smem = c.smem;
  const int tiles = (M + c.G - 1) / c.G * d.C;
  const float scale = 1.0f / ((float)d.H * (float)d.W);
  return launch_k(d.pdl, c.fn, tiles, threads, smem, stream, M, d.C, t.twH + col_tw_offset(idx), t.ax, t.by, scale,
                  spec);
}

}  // namespace ils
