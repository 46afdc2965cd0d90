// ILS hot-path kernels for sm_103a: one iteration of Algorithm 1 is
//   (1) row pass:    [inverse row FFT of u^n's row spectrum] -> Eq. 7 stencil and
//                    divergence -> right-hand side r = f + lambda/2 sum_* grad_*^T mu_*
//                    -> forward real row FFT -> packed row spectrum of r,
//   (2) column pass: column FFT -> divide by the Eq. 9 denominator -> inverse column FFT,
// and after the last iteration (3) an inverse real row FFT writes u^N.
// The numerator of Eq. 9 is formed in space: conj(F grad_*) F mu_* = F(grad_*^T mu_*)
// (Sec. 3.2), so each iteration needs one forward and one inverse 2-D FFT.
//
// Spectrum layout (per channel): H rows of M = W/2 complex values.  Slot k of
// row y holds X_y[k] (k = 1..M-1) of the row's real DFT; slot 0 holds the two
// real values (X_y[0], X_y[M]).  The buffer therefore has exactly the size of the
// image.  Column 0 is a pair of real sequences packed as one complex one and is
// divided in the column pass by separating the two halves through Hermitian
// symmetry.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>

#include "ils_fft.cuh"
#include "ils_internal.h"

namespace ils {


__device__ __forceinline__ int wrap_row(int y, int H) { return y < 0 ? y + H : (y >= H ? y - H : y); }

// ---------------------------------------------------------------- (1) fused row pass
// grid = (ceil(H / rows), C); each CTA produces `rows` rows of the r spectrum
// and needs u on rows y0-1 .. y0+rows (periodic), rebuilt from spec_in (or read
// from u0 / f on the first iteration).
template <int EPT, bool FIRST, int PEN>
__global__ void __launch_bounds__(512, EPT <= 16 ? 2 : 1)
row_forward_kernel(int H, int W, int rows, FftPlan planM, const float2* __restrict__ twW, MuParams mp,
                   const float* __restrict__ f, const float* __restrict__ u0,
                   const float2* __restrict__ spec_in, float2* __restrict__ spec_out,
                   float* __restrict__ u_ckpt) {
  griddep_launch();
  griddep_wait();
  extern __shared__ float2 sm[];
  const int M = W >> 1;
  const int ch = blockIdx.y;
  const int y0 = blockIdx.x * rows;
  const int nout = min(rows, H - y0);
  const int nin = nout + 2;
  const size_t plane = (size_t)H * M;  // complex (= float pairs) per channel
  const int T = blockDim.x;

  // 1. u^n on rows y0-1 .. y0+nout
  {
    const float2* src = FIRST ? reinterpret_cast<const float2*>(u0 ? u0 : f) + ch * plane
                              : spec_in + ch * plane;
    for (int w = threadIdx.x; w < nin * M; w += T) {
      const int i = w / M;
      const int m = w - i * M;
      const int yy = wrap_row(y0 - 1 + i, H);
      sm[smem_idx(w)] = src[(size_t)yy * M + m];
    }
    __syncthreads();
    if (!FIRST) {
      const int P = M / 2 + 1;
      for (int w = threadIdx.x; w < nin * P; w += T) {
        const int i = w / P;
        c2r_pre_pair(sm, i * M, M, w - i * P, twW);
      }
      __syncthreads();
      fft_smem<EPT, true>(sm, planM, nin, 1, M, twW, 2);
    }
  }
  if (u_ckpt != nullptr) {
    float2* dst = reinterpret_cast<float2*>(u_ckpt) + ch * plane + (size_t)y0 * M;
    for (int w = threadIdx.x; w < nout * M; w += T) dst[w] = sm[smem_idx(w + M)];
  }

  // 2. right-hand side r = f + lambda/2 (grad_x^T mu_x + grad_y^T mu_y), two pixels per item
  float2 rr[EPT];
  const float2* fc = reinterpret_cast<const float2*>(f) + ch * plane + (size_t)y0 * M;
#pragma unroll
  for (int b = 0; b < EPT; ++b) {
    const int w = threadIdx.x + b * T;
    if (w < nout * M && mp.half_lambda == 0.0f) {   // lambda = 0 (or a plain row FFT): r = f
      rr[b] = fc[w];
    } else if (w < nout * M) {
      const int i = w / M;
      const int m = w - i * M;
      const int ci = (i + 1) * M;
      const float2 c = sm[smem_idx(ci + m)];
      const float ul = sm[smem_idx(ci + (m == 0 ? M - 1 : m - 1))].y;
      const float ur = sm[smem_idx(ci + (m == M - 1 ? 0 : m + 1))].x;
      const float2 up = sm[smem_idx(i * M + m)];
      const float2 dn = sm[smem_idx((i + 2) * M + m)];
      const float2 fv = fc[w];
      const float mx_l = mu_pen<PEN>(c.x - ul, mp);    // mu_x at x0-1
      const float mx_c = mu_pen<PEN>(c.y - c.x, mp);   // mu_x at x0
      const float mx_r = mu_pen<PEN>(ur - c.y, mp);    // mu_x at x0+1
      const float my0u = mu_pen<PEN>(c.x - up.x, mp);  // mu_y at (y-1, x0)
      const float my0d = mu_pen<PEN>(dn.x - c.x, mp);  // mu_y at (y,   x0)
      const float my1u = mu_pen<PEN>(c.y - up.y, mp);
      const float my1d = mu_pen<PEN>(dn.y - c.y, mp);
      rr[b].x = fmaf(mp.half_lambda, (mx_l - mx_c) + (my0u - my0d), fv.x);
      rr[b].y = fmaf(mp.half_lambda, (mx_c - mx_r) + (my1u - my1d), fv.y);
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < EPT; ++b) {
    const int w = threadIdx.x + b * T;
    if (w < nout * M) sm[smem_idx(w)] = rr[b];
  }
  __syncthreads();

  // 3. forward real row FFT of r, packed, to spec_out
  fft_smem<EPT, false>(sm, planM, nout, 1, M, twW, 2);
  {
    const int P = M / 2 + 1;
    for (int w = threadIdx.x; w < nout * P; w += T) {
      const int i = w / P;
      r2c_post_pair(sm, i * M, M, w - i * P, twW);
    }
  }
  __syncthreads();
  float2* dst = spec_out + ch * plane + (size_t)y0 * M;
  for (int w = threadIdx.x; w < nout * M; w += T) dst[w] = sm[smem_idx(w)];
}

// ---------------------------------------------------------------- (2) column pass
// grid = (ceil(M / G), C); each CTA owns G whole complex columns.
template <int EPT>
__global__ void __launch_bounds__(512, EPT <= 16 ? 2 : 1)
col_solve_kernel(int H, int M, int G, FftPlan planH, const float2* __restrict__ twH,
                 const float* __restrict__ ax, const float* __restrict__ by, float scale,
                 float2* __restrict__ spec) {
  griddep_launch();
  griddep_wait();
  extern __shared__ float2 sm[];
  const int ch = blockIdx.y;
  const int k0 = blockIdx.x * G;
  const int g = min(G, M - k0);
  const int T = blockDim.x;
  float2* base = spec + (size_t)ch * H * M + k0;
  // element (column j, row y) at y*g + j
  for (int w = threadIdx.x; w < H * g; w += T) {
    const int y = w / g;
    sm[smem_idx(w)] = base[(size_t)y * M + (w - y * g)];
  }
  __syncthreads();
  fft_smem<EPT, false>(sm, planH, g, g, 1, twH, 1);

  // divide by den(l,k) = 1 + ax[k] + by[l] and scale by 1/(H W)  (Eq. 9)
  const int jstart = (k0 == 0) ? 1 : 0;
  for (int w = threadIdx.x; w < H * g; w += T) {
    const int l = w / g;
    const int j = w - l * g;
    if (j >= jstart) {
      const float s = __fdividef(scale, 1.0f + __ldg(&ax[k0 + j]) + __ldg(&by[l]));
      sm[smem_idx(w)] = cscale(sm[smem_idx(w)], s);
    }
  }
  if (k0 == 0) {
    // column 0 carries Z[l] = A[l] + i B[l] with A = F_y(X[:,0]), B = F_y(X[:,M]) (both Hermitian);
    // A/dA + i B/dB = Z[l] (1/dA + 1/dB)/2 + conj(Z[H-l]) (1/dA - 1/dB)/2.
    const float axM = __ldg(&ax[M]);
    for (int l = threadIdx.x; l <= H / 2; l += T) {
      const int lm = (l == 0) ? 0 : H - l;
      const float byl = __ldg(&by[l]);
      const float ia = __fdividef(1.0f, 1.0f + byl);
      const float ib = __fdividef(1.0f, 1.0f + axM + byl);
      const float sp = 0.5f * scale * (ia + ib);
      const float sn = 0.5f * scale * (ia - ib);
      const float2 zl = sm[smem_idx(l * g)];
      const float2 zm = sm[smem_idx(lm * g)];
      sm[smem_idx(l * g)] = make_float2(sp * zl.x + sn * zm.x, sp * zl.y - sn * zm.y);
      if (lm != l) sm[smem_idx(lm * g)] = make_float2(sp * zm.x + sn * zl.x, sp * zm.y - sn * zl.y);
    }
  }
  __syncthreads();
  fft_smem<EPT, true>(sm, planH, g, g, 1, twH, 1);
  for (int w = threadIdx.x; w < H * g; w += T) {
    const int y = w / g;
    base[(size_t)y * M + (w - y * g)] = sm[smem_idx(w)];
  }
}

// ---------------------------------------------------------------- adjoint row pass
// Reverse-mode step n of Algorithm 1 (not in the paper; the chain rule through Eq. 9 and Eq. 7).
// With A the Eq. 9 operator (symmetric: its Fourier eigenvalues are real and even) and
// gbar = dL/du^{n+1}: r = A^-1 gbar arrives as a row spectrum from the column pass.
//   fbar += r                                            (u^{n+1} depends on f linearly)
//   gbar' = lambda/2 sum_* grad_*^T [ g''(grad_* u^n) * grad_* r ]   (dL/du^n; g'' = dmu/dx, App. B)
// and gbar' is forward-FFT'd for the next step, or (last step) added to the u^0 gradient.
// g''(x) = c - p (x^2+eps)^(p/2-2) ((p-1) x^2 + eps).
// Welsch (Appendix B): g''(x) = c - 2 exp(-x^2/(2 gamma^2)) (1 - x^2/gamma^2).
template <int PEN>
__device__ __forceinline__ float g2_appb(float x, const MuParams& mp) {
  const float x2 = x * x;
  if constexpr (PEN == 1) {
    return fmaf(-2.0f * sfu_exp2(-mp.wbeta * x2), fmaf(-2.0f * mp.winv2g2, x2, 1.0f), mp.c);
  } else {
    const float t = x2 + mp.eps;
    const float w = sfu_exp2((mp.a - 1.0f) * sfu_log2(t));
    return fmaf(-mp.p * w, fmaf(mp.p - 1.0f, x2, mp.eps), mp.c);
  }
}

template <int EPT, int PEN>
__global__ void __launch_bounds__(512, EPT <= 16 ? 2 : 1)
row_adjoint_kernel(int H, int W, int rows, FftPlan planM, const float2* __restrict__ twW, MuParams mp,
                   const float2* __restrict__ spec_in, const float* __restrict__ u_n, float* __restrict__ fbar,
                   int fbar_first, float* __restrict__ gu0, int last, float2* __restrict__ spec_out) {
  griddep_launch();
  griddep_wait();
  extern __shared__ float2 sm[];
  const int M = W >> 1;
  const int ch = blockIdx.y;
  const int y0 = blockIdx.x * rows;
  const int nout = min(rows, H - y0);
  const int nin = nout + 2;
  const size_t plane = (size_t)H * M;
  const int T = blockDim.x;
  {
    const float2* src = spec_in + ch * plane;
    for (int w = threadIdx.x; w < nin * M; w += T) {
      const int i = w / M;
      const int m = w - i * M;
      sm[smem_idx(w)] = src[(size_t)wrap_row(y0 - 1 + i, H) * M + m];
    }
    __syncthreads();
    const int P = M / 2 + 1;
    for (int w = threadIdx.x; w < nin * P; w += T) {
      const int i = w / P;
      c2r_pre_pair(sm, i * M, M, w - i * P, twW);
    }
    __syncthreads();
    fft_smem<EPT, true>(sm, planM, nin, 1, M, twW, 2);
  }
  const float2* uc = reinterpret_cast<const float2*>(u_n) + ch * plane;
  float2* fb = reinterpret_cast<float2*>(fbar) + ch * plane;
  float2* g0 = gu0 ? reinterpret_cast<float2*>(gu0) + ch * plane : nullptr;
  float2 rr[EPT];
#pragma unroll
  for (int b = 0; b < EPT; ++b) {
    const int w = threadIdx.x + b * T;
    if (w < nout * M) {
      const int i = w / M;
      const int m = w - i * M;
      const int y = y0 + i;
      const int ml = m == 0 ? M - 1 : m - 1, mr = m == M - 1 ? 0 : m + 1;
      const int ci = (i + 1) * M;
      const float2 rc = sm[smem_idx(ci + m)];
      const float rl = sm[smem_idx(ci + ml)].y;
      const float rrt = sm[smem_idx(ci + mr)].x;
      const float2 ru = sm[smem_idx(i * M + m)];
      const float2 rd = sm[smem_idx((i + 2) * M + m)];
      const float2 uc0 = uc[(size_t)y * M + m];
      const float ul = uc[(size_t)y * M + ml].y;
      const float ur = uc[(size_t)y * M + mr].x;
      const float2 uu = uc[(size_t)wrap_row(y - 1, H) * M + m];
      const float2 ud = uc[(size_t)wrap_row(y + 1, H) * M + m];
      // q_x at x0-1, x0, x0+1 and q_y at (y-1, x) and (y, x)
      const float qx_l = g2_appb<PEN>(uc0.x - ul, mp) * (rc.x - rl);
      const float qx_c = g2_appb<PEN>(uc0.y - uc0.x, mp) * (rc.y - rc.x);
      const float qx_r = g2_appb<PEN>(ur - uc0.y, mp) * (rrt - rc.y);
      const float qy0u = g2_appb<PEN>(uc0.x - uu.x, mp) * (rc.x - ru.x);
      const float qy0d = g2_appb<PEN>(ud.x - uc0.x, mp) * (rd.x - rc.x);
      const float qy1u = g2_appb<PEN>(uc0.y - uu.y, mp) * (rc.y - ru.y);
      const float qy1d = g2_appb<PEN>(ud.y - uc0.y, mp) * (rd.y - rc.y);
      const float2 gb = make_float2(mp.half_lambda * ((qx_l - qx_c) + (qy0u - qy0d)),
                                    mp.half_lambda * ((qx_c - qx_r) + (qy1u - qy1d)));
      const size_t o = (size_t)y * M + m;
      float2 acc = fbar_first ? make_float2(0.f, 0.f) : fb[o];
      acc.x += rc.x;
      acc.y += rc.y;
      if (last && g0 == nullptr) {
        acc.x += gb.x;
        acc.y += gb.y;
      }
      fb[o] = acc;
      if (last && g0 != nullptr) g0[o] = gb;
      rr[b] = gb;
    }
  }
  if (last) return;   // block-uniform
  __syncthreads();
#pragma unroll
  for (int b = 0; b < EPT; ++b) {
    const int w = threadIdx.x + b * T;
    if (w < nout * M) sm[smem_idx(w)] = rr[b];
  }
  __syncthreads();
  fft_smem<EPT, false>(sm, planM, nout, 1, M, twW, 2);
  {
    const int P = M / 2 + 1;
    for (int w = threadIdx.x; w < nout * P; w += T) {
      const int i = w / P;
      r2c_post_pair(sm, i * M, M, w - i * P, twW);
    }
  }
  __syncthreads();
  float2* dst = spec_out + ch * plane + (size_t)y0 * M;
  for (int w = threadIdx.x; w < nout * M; w += T) dst[w] = sm[smem_idx(w)];
}

// ---------------------------------------------------------------- (3) final inverse row pass
template <int EPT, int EPI>
__global__ void __launch_bounds__(512, EPT <= 16 ? 2 : 1)
row_inverse_kernel(int H, int W, int rows, FftPlan planM, const float2* __restrict__ twW,
                   const float2* __restrict__ spec, float* __restrict__ u, Epilogue epi) {
  griddep_launch();
  griddep_wait();
  extern __shared__ float2 sm[];
  const int M = W >> 1;
  const int ch = blockIdx.y;
  const int y0 = blockIdx.x * rows;
  const int n = min(rows, H - y0);
  const size_t plane = (size_t)H * M;
  const int T = blockDim.x;
  const float2* src = spec + ch * plane + (size_t)y0 * M;
  for (int w = threadIdx.x; w < n * M; w += T) sm[smem_idx(w)] = src[w];
  __syncthreads();
  const int P = M / 2 + 1;
  for (int w = threadIdx.x; w < n * P; w += T) {
    const int i = w / P;
    c2r_pre_pair(sm, i * M, M, w - i * P, twW);
  }
  __syncthreads();
  fft_smem<EPT, true>(sm, planM, n, 1, M, twW, 2);
  const size_t rowoff = ch * plane + (size_t)y0 * M;
  float dm = 0.0f;
  for (int w = threadIdx.x; w < n * M; w += T)
    dm = fmaxf(dm, epi.template store<EPI>(reinterpret_cast<float2*>(u), rowoff + w, sm[smem_idx(w)]));
  epi.template finish<EPI>(dm);
}

// ---------------------------------------------------------------- host side

static int round_up(int a, int b) { return (a + b - 1) / b * b; }

bool make_fft_plan(int n, FftPlan* out) {
  if (n < 1) return false;
  FftPlan p{};
  p.n = n;
  int m = n, s = 0;
  auto push = [&](int r) {
    if (s >= kMaxStages) return false;
    p.radix[s++] = r;
    m /= r;
    return true;
  };
  while (m % 8 == 0) if (!push(8)) return false;
  while (m % 4 == 0) if (!push(4)) return false;
  while (m % 2 == 0) if (!push(2)) return false;
  while (m % 3 == 0) if (!push(3)) return false;
  while (m % 5 == 0) if (!push(5)) return false;
  if (m != 1) return false;
  p.nstages = s;
  *out = p;
  return true;
}

static constexpr int kMaxThreads = 512;
static constexpr size_t kSmemLimit = 200 * 1024;

// Smallest EPT in {16, 32} and a thread count (multiple of 32, 64..512) that
// cover `elems` complex values; false if even 32 x 512 does not.
static bool tile_config(int elems, int* ept, int* threads) {
  for (int e : {16, 32}) {
    if (elems <= e * kMaxThreads) {
      int t = round_up((elems + e - 1) / e, 32);
      const int want = round_up((elems + 11) / 12, 32);  // ~12 values per thread when possible
      if (t < want) t = want;
      if (t < 64) t = 64;
      if (t > kMaxThreads) t = kMaxThreads;
      *ept = e;
      *threads = t;
      return true;
    }
  }
  return false;
}

static bool fits(int elems) {
  return elems <= 32 * kMaxThreads && (size_t)smem_elems(elems) * sizeof(float2) <= kSmemLimit;
}

bool pick_geometry(int H, int W, Geometry* g) {
  const int M = W / 2;
  // fused row pass: rows + 2 rows of M complex; prefer a tile that runs two CTAs per SM
  int rows = 0;
  for (int r = 8; r >= 1; --r) {
    if ((r + 2) * M <= 16 * kMaxThreads && (size_t)smem_elems((r + 2) * M) * 8 <= kSmemLimit / 2) { rows = r; break; }
  }
  if (rows == 0)
    for (int r = 8; r >= 1; --r) if (fits((r + 2) * M)) { rows = r; break; }
  if (rows == 0) return false;
  if (rows > H) rows = H;
  g->rows_fwd = rows;
  if (!tile_config((rows + 2) * M, &g->ept_row, &g->threads_row)) return false;
  g->smem_fwd = (size_t)smem_elems((rows + 2) * M) * sizeof(float2);
  int ri = 0;
  for (int r = 8; r >= 1; --r) if (r * M <= 16 * kMaxThreads) { ri = r; break; }
  if (ri == 0) ri = 1;
  if (ri > H) ri = H;
  if (!fits(ri * M) || !tile_config(ri * M, &g->ept_inv, &g->threads_inv)) return false;
  g->rows_inv = ri;
  g->smem_inv = (size_t)smem_elems(ri * M) * sizeof(float2);
  // column pass: G whole columns of H complex; G >= 4 keeps 32-byte sectors whole
  int G = 0;
  for (int c = 16; c >= 1; c >>= 1) {
    if (c > M && c > 1) continue;
    if (fits(H * c) && (c <= 4 || H * c <= 16 * kMaxThreads)) { G = c; break; }
  }
  if (G == 0 || !tile_config(H * G, &g->ept_col, &g->threads_col)) return false;
  g->cols = G;
  g->smem_col = (size_t)smem_elems(H * G) * sizeof(float2);
  // Compile-time plans where one exists; ILS_FORCE_GENERIC=1 keeps the generic kernels
  // (used by the tests to cover both implementations on the same sizes).
  // ILS_ROW_IMPL=fixed|generic selects the block-per-strip or generic row kernels instead
  // of the warp-per-row ones, ILS_ROW_IMPL=warp<k> the k-th warp-per-row variant of the
  // length (tests compare the implementations on the same sizes).
  const char* force = getenv("ILS_FORCE_GENERIC");
  const bool generic = force != nullptr && force[0] == '1';
  const char* impl = getenv("ILS_ROW_IMPL");
  const bool no_warp = generic || (impl != nullptr && (impl[0] == 'f' || impl[0] == 'g'));
  const bool no_fixed = generic || (impl != nullptr && impl[0] == 'g');
  int wv[8];
  const int nw = no_warp ? 0 : warp_row_variants(M, wv, 8);
  int pick = 0;
  if (impl != nullptr && impl[0] == 'w' && impl[1] == 'a' && impl[2] == 'r' && impl[3] == 'p') {
    pick = atoi(impl + 4);
    if (pick < 0 || pick >= nw) pick = 0;
  }
  g->warp_row = nw > 0 ? wv[pick] : -1;
  g->warp_adj = g->warp_row >= 0 && warp_row_has_adjoint(g->warp_row) ? g->warp_row : -1;
  g->fixed_row = no_fixed ? -1 : fixed_row_index(M);
  // 256-wide rows (M = 128): the block-per-strip plan by default.  A warp-per-row transform of
  // 4 points per lane runs its 32-point stage on 4 of the 32 lanes; measured on a 48 x 256 x 256
  // call: 158 us per call against 181 us (row pass 27.5 against 34.8 us, final inverse 12.4
  // against 18.3 us).  The adjoint keeps its warp-per-row kernel.
  if (impl == nullptr && M == 128 && g->fixed_row >= 0) g->warp_row = -1;
  // ILS_ROW_IMPL=fixed<k>: the k-th compile-time row plan of the length
  if (!no_fixed && impl != nullptr && impl[0] == 'f' && impl[1] == 'i' && impl[2] == 'x' && impl[3] == 'e' &&
      impl[4] == 'd' && impl[5] >= '0' && impl[5] <= '9') {
    int rv[16];
    const int nr = fixed_row_variants(M, rv, 16);
    const int k = atoi(impl + 5);
    if (k >= 0 && k < nr) g->fixed_row = rv[k];
  }
  g->fixed_col = generic ? -1 : fixed_col_index(H);
  // ILS_COL_IMPL=<k>: the k-th compile-time column plan of the length (tests, measurements)
  const char* cimpl = getenv("ILS_COL_IMPL");
  if (!generic && cimpl != nullptr && cimpl[0] >= '0' && cimpl[0] <= '9') {
    int cv[16];
    const int nc = fixed_col_variants(H, cv, 16);
    const int k = atoi(cimpl);
    if (k >= 0 && k < nc) g->fixed_col = cv[k];
  }
  return true;
}

template <typename K>
static cudaError_t allow_smem(K kernel) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit);
}

cudaError_t set_kernel_attributes() {
  cudaError_t e;
  if ((e = allow_smem(row_forward_kernel<16, true, 0>))) return e;
  if ((e = allow_smem(row_forward_kernel<16, false, 0>))) return e;
  if ((e = allow_smem(row_forward_kernel<32, true, 0>))) return e;
  if ((e = allow_smem(row_forward_kernel<32, false, 0>))) return e;
  if ((e = allow_smem(row_forward_kernel<16, true, 1>))) return e;
  if ((e = allow_smem(row_forward_kernel<16, false, 1>))) return e;
  if ((e = allow_smem(row_forward_kernel<32, true, 1>))) return e;
  if ((e = allow_smem(row_forward_kernel<32, false, 1>))) return e;
  if ((e = allow_smem(row_forward_kernel<16, true, 2>))) return e;
  if ((e = allow_smem(row_forward_kernel<16, false, 2>))) return e;
  if ((e = allow_smem(row_forward_kernel<32, true, 2>))) return e;
  if ((e = allow_smem(row_forward_kernel<32, false, 2>))) return e;
  if ((e = allow_smem(col_solve_kernel<16>))) return e;
  if ((e = allow_smem(col_solve_kernel<32>))) return e;
  if ((e = allow_smem(row_inverse_kernel<16, 0>))) return e;
  if ((e = allow_smem(row_inverse_kernel<32, 0>))) return e;
  if ((e = allow_smem(row_inverse_kernel<16, 1>))) return e;
  if ((e = allow_smem(row_inverse_kernel<32, 1>))) return e;
  if ((e = allow_smem(row_inverse_kernel<16, 2>))) return e;
  if ((e = allow_smem(row_inverse_kernel<32, 2>))) return e;
  if ((e = allow_smem(row_inverse_kernel<16, 3>))) return e;
  if ((e = allow_smem(row_inverse_kernel<32, 3>))) return e;
  if ((e = allow_smem(row_inverse_kernel<16, 4>))) return e;
  if ((e = allow_smem(row_inverse_kernel<32, 4>))) return e;
  if ((e = allow_smem(row_inverse_kernel<16, 5>))) return e;
  if ((e = allow_smem(row_inverse_kernel<32, 5>))) return e;
  if ((e = allow_smem(row_adjoint_kernel<16, 0>))) return e;
  if ((e = allow_smem(row_adjoint_kernel<32, 0>))) return e;
  if ((e = allow_smem(row_adjoint_kernel<16, 1>))) return e;
  if ((e = allow_smem(row_adjoint_kernel<32, 1>))) return e;
  if ((e = warp_set_attributes())) return e;
  return fixed_set_attributes();
}

cudaError_t launch_row_forward(const ImageDesc& d, const Geometry& g, const Tables& t, const MuParams& mp,
                               const float* f, const float* u0, const float2* spec_in, float2* spec_out,
                               float* u_ckpt, cudaStream_t stream) {
  if (g.warp_row >= 0) return warp_row_forward(g.warp_row, d, t, mp, f, u0, spec_in, spec_out, u_ckpt, stream);
  if (g.fixed_row >= 0) return fixed_row_forward(g.fixed_row, d, t, mp, f, u0, spec_in, spec_out, u_ckpt, stream);
  dim3 grid((d.H + g.rows_fwd - 1) / g.rows_fwd, d.C);
  const int T = g.threads_row;
  const size_t S = g.smem_fwd;
  const bool first = spec_in == nullptr;
  using Fn = decltype(&row_forward_kernel<16, true, 0>);
  static const Fn table[kPenalties][2][2] = {
      {{row_forward_kernel<16, true, 0>, row_forward_kernel<16, false, 0>},
       {row_forward_kernel<32, true, 0>, row_forward_kernel<32, false, 0>}},
      {{row_forward_kernel<16, true, 1>, row_forward_kernel<16, false, 1>},
       {row_forward_kernel<32, true, 1>, row_forward_kernel<32, false, 1>}},
      {{row_forward_kernel<16, true, 2>, row_forward_kernel<16, false, 2>},
       {row_forward_kernel<32, true, 2>, row_forward_kernel<32, false, 2>}}};
  Fn fn = table[mp.pen][g.ept_row == 16 ? 0 : 1][first ? 0 : 1];
  return launch_k(d.pdl, fn, grid, T, S, stream, d.H, d.W, g.rows_fwd, d.planM, t.twW, mp, f, first ? u0 : nullptr,
                  spec_in, spec_out, u_ckpt);
}

cudaError_t launch_col_solve(const ImageDesc& d, const Geometry& g, const Tables& t, float2* spec,
                             cudaStream_t stream) {
  if (g.fixed_col >= 0) return fixed_col_solve(g.fixed_col, d, t, spec, stream);
  const int M = d.W / 2;
  dim3 grid((M + g.cols - 1) / g.cols, d.C);
  const float scale = 1.0f / ((float)d.H * (float)d.W);
  auto fn = g.ept_col == 16 ? col_solve_kernel<16> : col_solve_kernel<32>;
  return launch_k(d.pdl, fn, grid, g.threads_col, g.smem_col, stream, d.H, M, g.cols, d.planH, t.twH, t.ax, t.by, scale,
                  spec);
}

cudaError_t launch_row_inverse(const ImageDesc& d, const Geometry& g, const Tables& t, const float2* spec,
                               float* u, cudaStream_t stream, const Epilogue& epi) {
  if (g.warp_row >= 0) return warp_row_inverse(g.warp_row, d, t, spec, u, stream, epi);
  if (g.fixed_row >= 0) return fixed_row_inverse(g.fixed_row, d, t, spec, u, stream, epi);
  dim3 grid((d.H + g.rows_inv - 1) / g.rows_inv, d.C);
  using InvFn = void (*)(int, int, int, FftPlan, const float2*, const float2*, float*, Epilogue);
  static const InvFn fns[2][kEpilogues] = {
      {row_inverse_kernel<16, 0>, row_inverse_kernel<16, 1>, row_inverse_kernel<16, 2>, row_inverse_kernel<16, 3>,
       row_inverse_kernel<16, 4>, row_inverse_kernel<16, 5>},
      {row_inverse_kernel<32, 0>, row_inverse_kernel<32, 1>, row_inverse_kernel<32, 2>, row_inverse_kernel<32, 3>,
       row_inverse_kernel<32, 4>, row_inverse_kernel<32, 5>}};
  const InvFn fn = fns[g.ept_inv == 16 ? 0 : 1][epi.mode];
  return launch_k(d.pdl, fn, grid, g.threads_inv, g.smem_inv, stream, d.H, d.W, g.rows_inv, d.planM, t.twW, spec, u,
                  epi);
}

cudaError_t launch_row_adjoint(const ImageDesc& d, const Geometry& g, const Tables& t, const MuParams& mp,
                               const float2* spec_in, const float* u_n, float* fbar, bool fbar_first, float* gu0,
                               bool last, float2* spec_out, cudaStream_t stream) {
  if (mp.pen == 2) return cudaErrorInvalidValue;  // no adjoint for half-quadratic splitting
  if (g.warp_adj >= 0)
    return warp_row_adjoint(g.warp_adj, d, t, mp, spec_in, u_n, fbar, fbar_first, gu0, last, spec_out, stream);
  dim3 grid((d.H + g.rows_fwd - 1) / g.rows_fwd, d.C);
  auto fn = mp.pen == 1 ? (g.ept_row == 16 ? row_adjoint_kernel<16, 1> : row_adjoint_kernel<32, 1>)
                      : (g.ept_row == 16 ? row_adjoint_kernel<16, 0> : row_adjoint_kernel<32, 0>);
  return launch_k(d.pdl, fn, grid, g.threads_row, g.smem_fwd, stream, d.H, d.W, g.rows_fwd, d.planM, t.twW, mp, spec_in,
                  u_n, fbar, (int)fbar_first, gu0, (int)last, spec_out);
}

}  // namespace ils
