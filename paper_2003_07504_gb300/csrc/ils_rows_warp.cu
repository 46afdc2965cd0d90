// Row passes with one warp per image row, for row lengths W = 64 L (M = W/2 = 32 L complex),
// and with a warp pair per row for W = 128 L (PairRow below).
//
// A warp transforms one packed complex row of M = 32 L points as a 32 x L four-step FFT:
// lane n1 holds x[n1 + 32 n2] (n2 = 0..L-1, a coalesced row load), runs the L-point DFT
// over its registers (ils_dft.cuh), multiplies by w_M^{n1 k2}, and the warp transposes
// through its own shared-memory row buffer (stride 33, conflict free) so that lane k2 < L
// holds the 32 values of index k2 and runs the 32-point DFT: X[k2 + L k1] lands in
// register k1 of lane k2.  The only barriers inside a transform are __syncwarp.
//
// The fused row pass of iteration n (see ils_kernels.cu for the passes and the packed
// spectrum layout) then needs two CTA barriers per strip: after the inverse transforms of
// the ROWS + 2 rows (the stencil reads neighbouring rows) and after the stencil (a row's
// buffer is reused by its forward transform).
#include <cuda_runtime.h>

#include "ils_dft.cuh"
#include "ils_internal.h"

namespace ils {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int wrap_row(int y, int H) { return y < 0 ? y + H : (y >= H ? y - H : y); }

// 16-byte asynchronous global -> shared copies (cp.async; completion waited per thread).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(__cvta_generic_to_global(gmem)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// waits until at most N of this thread's committed copy groups are still in flight
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}


// Twiddle tables of a row transform: rt[k] = exp(-2 pi i k / (2M)) for k < M (the real-FFT
// packing and unpacking) and ft[32 k2 + n1] = exp(-2 pi i n1 k2 / M) (the four-step twiddles,
// k2-major so a warp reads 32 consecutive entries).  Either straight from the global table
// (Tables::twW: rt = twW, ft = twW + 2M) or from a CTA's shared-memory copy (stage_row_twiddles:
// rt = tws, ft = tws + M), which turns the transforms' dependent global loads into
// shared-memory loads.
struct TwRef {
  const float2* rt;
  const float2* ft;
};

// CTA-wide 16-byte asynchronous copy of the row twiddles into tws[0 .. 2M) (rt then ft); the
// caller waits (cp.async.wait_all) and synchronizes the CTA before the first use.
template <int M>
__device__ __forceinline__ void stage_row_twiddles(float2* tws, const float2* __restrict__ twW) {
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    const int part = i >= M / 2 ? 1 : 0, c = i - part * (M / 2);
    cp_async16(tws + part * M + 2 * c, twW + part * 2 * M + 2 * c);
  }
}

template <int L>
struct WarpRow {
  static constexpr int M = 32 * L;
  static constexpr int STRIDE = 33;                       // complex per transposed line
  static constexpr int BUF = (L * STRIDE > M ? L * STRIDE : M);  // complex per row buffer

  static constexpr int K2P = (L + 31) / 32;  // 32-point transforms per lane (k2 = lane + 32 j < L)

  // v: lane holds x[lane + 32 n2]; out[j] (where k2 = lane + 32 j < L): X[k2 + L k1].  buf: this
  // warp's buffer.  L > 32 (a 1920-point row) runs two 32-point transforms per lane.
  template <bool INV>
  __device__ __forceinline__ static void fft(float2 (&v)[L], float2 (&out)[K2P][32], float2* buf, int lane,
                                             const TwRef& tw) {
    dft_reg<L, INV>(v);
#pragma unroll
    for (int k2 = 1; k2 < L; ++k2) {
      float2 w = tw.ft[32 * k2 + lane];  // w_M^{lane k2}
      if (INV) w.y = -w.y;
      v[k2] = cmul(v[k2], w);
    }
#pragma unroll
    for (int k2 = 0; k2 < L; ++k2) buf[k2 * STRIDE + lane] = v[k2];
    __syncwarp();
#pragma unroll
    for (int j = 0; j < K2P; ++j) {
      const int k2 = lane + 32 * j;
      if (k2 < L) {
#pragma unroll
        for (int n1 = 0; n1 < 32; ++n1) out[j][n1] = buf[k2 * STRIDE + n1];
        dft_reg<32, INV>(out[j]);
      }
    }
    __syncwarp();
  }

  // 16-byte asynchronous copy of the packed spectrum row X into buf (the caller waits).
  __device__ __forceinline__ static void stage_row(const float2* __restrict__ X, float2* buf, int lane) {
    static_assert(L % 2 == 0, "16-byte copies of a 32 L-point row need L even");
#pragma unroll
    for (int q = 0; q < L / 2; ++q) cp_async16(buf + 2 * (lane + 32 * q), X + 2 * (lane + 32 * q));
  }

  // Hermitian unpacking of the packed half spectrum X for the inverse real transform:
  // v[n2] = Z[k], k = lane + 32 n2, with Z[k] = (X[k] + conj X[M-k]) + i e^{+2 pi i k/(2M)}
  // (X[k] - conj X[M-k]) and Z[0] from slot 0 = (X[0], X[M]).  X is a global row, or the row
  // staged in this warp's buffer (stage_row; then every lane has read buf on return).
  template <bool STAGED>
  __device__ __forceinline__ static void load_c2r(const float2* __restrict__ X, float2 (&v)[L], float2* buf, int lane,
                                                  const TwRef& tw) {
    const float2* src = STAGED ? buf : X;
#pragma unroll
    for (int n2 = 0; n2 < L; ++n2) {
      const int k = lane + 32 * n2;
      if (k == 0) {
        const float2 x = src[0];
        v[n2] = c2(x.x + x.y, x.x - x.y);
      } else {
        const float2 a = src[k], b = cconj(src[M - k]);
        const float2 s = cadd(a, b), d = csub(a, b);
        const float2 t = cmul(cconj(tw.rt[k]), d);
        v[n2] = c2(s.x - t.y, s.y + t.x);
      }
    }
    if (STAGED) __syncwarp();  // every lane has read buf before the transform writes it
  }

  // Inverse real transform of the packed half spectrum X (global row, or staged in buf) into
  // buf in natural order: buf[m] = (x[2m], x[2m+1]) * (the unnormalized factor 2M; the column
  // pass divides).
  template <bool STAGED>
  __device__ __forceinline__ static void inverse_row_to_buf(const float2* __restrict__ X, float2* buf, int lane,
                                                            const TwRef& tw) {
    float2 v[L];
    load_c2r<STAGED>(X, v, buf, lane, tw);
    float2 out[K2P][32];
    fft<true>(v, out, buf, lane, tw);
#pragma unroll
    for (int j = 0; j < K2P; ++j) {
      if (lane + 32 * j < L) {
#pragma unroll
        for (int k1 = 0; k1 < 32; ++k1) buf[lane + 32 * j + L * k1] = out[j][k1];
      }
    }
    __syncwarp();
  }

  // Inverse real transform of X (global row, or staged in buf) straight to global memory
  // through the epilogue (pair index rowoff + m of the output image).
  template <int EPI, bool STAGED>
  __device__ __forceinline__ static void inverse_row_to_global(const float2* __restrict__ X, float2* out,
                                                               size_t rowoff, const Epilogue& epi, float2* buf,
                                                               int lane, const TwRef& tw) {
    float2 v[L];
    load_c2r<STAGED>(X, v, buf, lane, tw);
    float2 res[K2P][32];
    fft<true>(v, res, buf, lane, tw);
    float dm = 0.0f;
#pragma unroll
    for (int j = 0; j < K2P; ++j) {
      if (lane + 32 * j < L) {
#pragma unroll
        for (int k1 = 0; k1 < 32; ++k1)
          dm = fmaxf(dm, epi.template store<EPI>(out, rowoff + lane + 32 * j + L * k1, res[j][k1]));
      }
    }
    epi.template finish<EPI>(dm);
  }

  // Forward real transform of r (lane holds r-pairs at m = lane + 32 n2) to the packed
  // half spectrum in the global row dst (slot 0 = (X[0], X[M])).
  __device__ __forceinline__ static void forward_row_to_global(float2 (&v)[L], float2* dst, float2* buf, int lane,
                                                               const TwRef& tw) {
    float2 out[K2P][32];
    fft<false>(v, out, buf, lane, tw);
#pragma unroll
    for (int j = 0; j < K2P; ++j) {
      if (lane + 32 * j < L) {
#pragma unroll
        for (int k1 = 0; k1 < 32; ++k1) buf[lane + 32 * j + L * k1] = out[j][k1];
      }
    }
    __syncwarp();
    pack_to_global(buf, dst, lane, tw);
  }

  // buf holds Z = FFT_M(r[2m] + i r[2m+1]) in natural order: write the packed half spectrum
  // of the real row r to dst, pairs (k, M-k) for k = 0..M/2.
  __device__ __forceinline__ static void pack_to_global(const float2* buf, float2* dst, int lane, const TwRef& tw) {
#pragma unroll
    for (int q = 0; q < (M / 2 + 1 + 31) / 32; ++q) {
      const int k = lane + 32 * q;
      if (k > M / 2) continue;
      if (k == 0) {
        const float2 z = buf[0];
        dst[0] = c2(z.x + z.y, z.x - z.y);
      } else {
        const float2 a = buf[k], b = buf[M - k];
        const float2 fa = cscale(cadd(a, cconj(b)), 0.5f), fo = cscale(csub(a, cconj(b)), 0.5f);
        dst[k] = cadd(fa, cmul(tw.rt[k], c2(fo.y, -fo.x)));
        if (M - k != k) {
          const float2 fb = cscale(cadd(b, cconj(a)), 0.5f), fq = cscale(csub(b, cconj(a)), 0.5f);
          dst[M - k] = cadd(fb, cmul(tw.rt[M - k], c2(fq.y, -fq.x)));
        }
      }
    }
    __syncwarp();
  }
};

// The shared-mu stencil (Eq. 7 and the divergence of Eq. 9's numerator) of a row-pass CTA,
// each mu evaluated once; every thread of the CTA calls it (three CTA barriers).  On entry
// strip row b (rows y0-1 .. y0+nout) is in buffer b in natural pair order; on return output
// warp w = o+1 (out_live) holds r of output row o in v (lane: pairs m = lane + 32 n2), and
// buffer w-1 has no other reader left (its scratch for the forward transform).
//   fr:  global f row of output row o (read when neither staged nor equal to u);
//   fst: staged f row (STAGE); f_is_u: f equals u^n (the first pass from u^0 = f);
//   ck:  checkpoint row of output row o or null (receives u^n).
template <int L, bool STAGE, int PEN>
__device__ __forceinline__ void stencil_shared(float2 (&v)[L], const MuParams& mp, float2* sm, int w, int lane,
                                               int nout, bool out_live, bool f_is_u, const float2* fr,
                                               const float2* fst, float2* ck) {
  using WR = WarpRow<L>;
  auto U = [&](int row, int m) -> float2 { return sm[row * WR::BUF + m]; };
  float2* buf = sm + w * WR::BUF;
  // S1: warp b <= nout computes mu_y at the boundary between strip rows b and b+1.
  float2 Y[L];
  if (w <= nout) {
#pragma unroll
    for (int n2 = 0; n2 < L; ++n2) {
      const int m = lane + 32 * n2;
      const float2 a = U(w, m), b = U(w + 1, m);
      Y[n2] = c2(mu_pen<PEN>(b.x - a.x, mp), mu_pen<PEN>(b.y - a.y, mp));
    }
  }
  if (STAGE) cp_async_wait_all();
  __syncthreads();
  // S2: an output warp forms r = f + lambda/2 (div_x mu_x - mu_y(own boundary)) from its own
  // row, mu_x once per pixel; x neighbours move between lanes by shuffle, so each lane reads
  // and then overwrites only its own pairs (mu_y of its boundary replaces u in place).
  if (w <= nout) {
    float2 cn = buf[lane];
    const float u_first = __shfl_sync(kFull, cn.x, 0);  // pixel 0: right neighbour of pixel 2M-1
    float carry = 0.0f;  // mu_x of the pixel left of lane 0's pair
#pragma unroll
    for (int n2 = 0; n2 < L; ++n2) {
      const int m = lane + 32 * n2;
      const float2 c = cn;
      if (n2 + 1 < L) cn = buf[m + 32];
      if (out_live) {
        const float nx_in = __shfl_down_sync(kFull, c.x, 1);
        const float nx_wrap = __shfl_sync(kFull, n2 + 1 < L ? cn.x : u_first, 0);
        const float nx = lane == 31 ? nx_wrap : nx_in;  // u at pixel 2m+2
        const float mx_c = mu_pen<PEN>(c.y - c.x, mp);     // mu_x at pixel 2m
        const float mx_r = mu_pen<PEN>(nx - c.y, mp);      // mu_x at pixel 2m+1
        const float up = __shfl_up_sync(kFull, mx_r, 1);
        const float mx_l = lane == 0 ? carry : up;    // mu_x at pixel 2m-1
        carry = __shfl_sync(kFull, mx_r, 31);
        const float2 fv = f_is_u ? c : (STAGE ? fst[m] : fr[m]);
        v[n2] = c2(fmaf(mp.half_lambda, (mx_l - mx_c) - Y[n2].x, fv.x),
                   fmaf(mp.half_lambda, (mx_c - mx_r) - Y[n2].y, fv.y));
        if (ck != nullptr) ck[m] = c;
      }
      buf[m] = Y[n2];
    }
    // lane 0's first pair: the left neighbour of pixel 0 is pixel 2M-1, finished last
    if (out_live && lane == 0) v[0].x = fmaf(mp.half_lambda, carry, v[0].x);
  }
  __syncthreads();
  // S3: add mu_y of the boundary above (written by warp w-1); that row buffer has no other
  // reader now, so it becomes this warp's scratch for the forward transform.
  if (out_live) {
    const float2* above = sm + (w - 1) * WR::BUF;
#pragma unroll
    for (int n2 = 0; n2 < L; ++n2) {
      const float2 t = above[lane + 32 * n2];
      v[n2] = c2(fmaf(mp.half_lambda, t.x, v[n2].x), fmaf(mp.half_lambda, t.y, v[n2].y));
    }
    __syncwarp();
  }
}

// Copies the u^0 rows of a first row pass into the strip buffers (16-byte asynchronous copies
// when the row is 16-byte aligned; the caller waits and synchronizes).
template <int L>
__device__ __forceinline__ void load_u0_row(const float2* __restrict__ src, float2* buf, int lane) {
  if (L % 2 == 0 && (reinterpret_cast<size_t>(src) & 15) == 0) {
#pragma unroll
    for (int q = 0; q < L / 2; ++q) cp_async16(buf + 2 * (lane + 32 * q), src + 2 * (lane + 32 * q));
  } else {
#pragma unroll
    for (int n2 = 0; n2 < L; ++n2) buf[lane + 32 * n2] = src[lane + 32 * n2];
  }
}

// Fused row pass: CTA = ROWS + 2 warps over rows y0-1 .. y0+ROWS (periodic); warp w holds
// strip row w in buffer w.  FIRST: u^0 rows are read from u0 (or f); otherwise rebuilt by the
// inverse transform of spec_in.  Then warp o+1 computes r for output row o and transforms it.
// SHARED: each mu is evaluated once (stencil_shared); otherwise every warp evaluates the mu
// of all four gradients of each of its pixels and of the left neighbour (two barriers, no
// cross-warp data beyond the strip rows).
// STAGE (with SHARED): the f rows of the output rows are copied to shared memory
// asynchronously at the start (behind the inverse transforms) instead of being loaded in
// the stencil; not when f is the u^0 of a first pass (the strip rows already hold it).
template <int L, int ROWS, bool FIRST, bool STAGE, bool SHARED, int PEN, int MINB, bool SPEC>
__global__ void __launch_bounds__((ROWS + 2) * 32, MINB)
row_warp_fwd_kernel(int H, const float2* __restrict__ twW, MuParams mp, const float* __restrict__ f,
                    const float* __restrict__ u0, const float2* __restrict__ spec_in, float2* __restrict__ spec_out,
                    float* __restrict__ u_ckpt) {
  griddep_launch();
  using WR = WarpRow<L>;
  constexpr int M = WR::M;
  extern __shared__ float2 sm[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int strips = (H + ROWS - 1) / ROWS;
  const int ch = blockIdx.x / strips;
  const int y0 = (blockIdx.x - ch * strips) * ROWS;
  const int nout = min(ROWS, H - y0);
  const size_t plane = (size_t)H * M;
  float2* buf = sm + w * WR::BUF;
  auto U = [&](int row, int m) -> float2 { return sm[row * WR::BUF + m]; };
  const int o = w - 1;  // output row of this warp
  const bool out_live = o >= 0 && o < nout;
  const bool f_is_u = FIRST && (u0 == nullptr || u0 == f);  // r's f term is the strip row itself
  const size_t orow = ch * plane + (size_t)(y0 + max(o, 0)) * M;  // pair offset of the output row
  float2* fst = sm + (ROWS + 2) * WR::BUF + max(o, 0) * M;  // staged f row (STAGE)
  float2* tws = sm + (ROWS + 2) * WR::BUF + (STAGE ? ROWS * M : 0);  // the CTA's twiddle tables
  const TwRef tw{tws, tws + M};
  stage_row_twiddles<M>(tws, twW);  // constant tables: before the wait on the previous grid
  griddep_wait();  // f is never written by this library's kernels; the spectrum is
  float2 v[L];
  const int yy = wrap_row(y0 - 1 + w, H);
  if (w < nout + 2) {
    if (FIRST) load_u0_row<L>(reinterpret_cast<const float2*>(u0 != nullptr ? u0 : f) + ch * plane + (size_t)yy * M,
                              buf, lane);
    else if (SPEC) WR::stage_row(spec_in + ch * plane + (size_t)yy * M, buf, lane);
  }
  cp_async_commit();
  if (STAGE && out_live && mp.half_lambda != 0.0f && !f_is_u) {  // waited for in the stencil
    const float2* src = reinterpret_cast<const float2*>(f) + orow;
    if ((reinterpret_cast<size_t>(src) & 15) == 0) {
#pragma unroll
      for (int q = 0; q < M / 64; ++q) cp_async16(fst + 2 * (lane + 32 * q), src + 2 * (lane + 32 * q));
    } else {
#pragma unroll
      for (int n2 = 0; n2 < L; ++n2) fst[lane + 32 * n2] = src[lane + 32 * n2];
    }
  }
  cp_async_commit();
  cp_async_wait_group<1>();  // the twiddles and this thread's strip-row copies have landed
  __syncthreads();
  if (!FIRST && w < nout + 2) WR::template inverse_row_to_buf<SPEC>(spec_in + ch * plane + (size_t)yy * M, buf, lane, tw);
  __syncthreads();
  if (mp.half_lambda == 0.0f) {  // lambda = 0 (or a plain row FFT): r = f
    if (out_live) {
      const float2* fr = reinterpret_cast<const float2*>(f) + orow;
#pragma unroll
      for (int n2 = 0; n2 < L; ++n2) {
        const int m = lane + 32 * n2;
        v[n2] = fr[m];
        if (u_ckpt != nullptr) reinterpret_cast<float2*>(u_ckpt)[orow + m] = U(w, m);
      }
      WR::forward_row_to_global(v, spec_out + orow, buf, lane, tw);
    }
    return;
  }
  if constexpr (!SHARED) {
    // Stencil (Eq. 7 and the divergence of Eq. 9's numerator) per pixel pair from the
    // strip rows alone: mu of the pair's three x gradients and four y gradients; the x
    // gradient left of a pair is the left lane's right one (shuffle; lane 0 takes lane 31's
    // from the previous block of 32 pairs, and pixel 0's wrap-around term is added last).
    if (out_live) {
      const float2* fr = reinterpret_cast<const float2*>(f) + orow;
      float carry = 0.0f;
#pragma unroll
      for (int n2 = 0; n2 < L; ++n2) {
        const int m = lane + 32 * n2;
        const float2 c = U(w, m);
        const float ur = U(w, m == M - 1 ? 0 : m + 1).x;
        const float2 up = U(w - 1, m);
        const float2 dn = U(w + 1, m);
        const float2 fv = f_is_u ? c : fr[m];
        const float mx_c = mu_pen<PEN>(c.y - c.x, mp);
        const float mx_r = mu_pen<PEN>(ur - c.y, mp);
        const float left = __shfl_up_sync(kFull, mx_r, 1);
        const float mx_l = lane == 0 ? carry : left;
        carry = __shfl_sync(kFull, mx_r, 31);
        const float my0u = mu_pen<PEN>(c.x - up.x, mp);
        const float my0d = mu_pen<PEN>(dn.x - c.x, mp);
        const float my1u = mu_pen<PEN>(c.y - up.y, mp);
        const float my1d = mu_pen<PEN>(dn.y - c.y, mp);
        v[n2] = c2(fmaf(mp.half_lambda, (mx_l - mx_c) + (my0u - my0d), fv.x),
                   fmaf(mp.half_lambda, (mx_c - mx_r) + (my1u - my1d), fv.y));
        if (u_ckpt != nullptr) reinterpret_cast<float2*>(u_ckpt)[orow + m] = c;
      }
      // pixel 0's left neighbour is pixel 2M-1, whose x gradient is the last carry
      if (lane == 0) v[0].x = fmaf(mp.half_lambda, carry, v[0].x);
    }
    __syncthreads();
    if (out_live) WR::forward_row_to_global(v, spec_out + orow, buf, lane, tw);
    return;
  } else {
    stencil_shared<L, STAGE, PEN>(v, mp, sm, w, lane, nout, out_live, f_is_u,
                                  reinterpret_cast<const float2*>(f) + orow, fst,
                                  u_ckpt != nullptr ? reinterpret_cast<float2*>(u_ckpt) + orow : nullptr);
    if (out_live) WR::forward_row_to_global(v, spec_out + orow, sm + (w - 1) * WR::BUF, lane, tw);
  }
}

// Final inverse row pass: one warp per row, ROWS rows per CTA; EPI: the epilogue mode.
template <int L, int ROWS, int EPI, bool SPEC>
__global__ void __launch_bounds__(ROWS * 32)
row_warp_inv_kernel(int H, const float2* __restrict__ twW, const float2* __restrict__ spec, float* __restrict__ u,
                    Epilogue epi) {
  griddep_launch();
  using WR = WarpRow<L>;
  constexpr int M = WR::M;
  extern __shared__ float2 sm[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int strips = (H + ROWS - 1) / ROWS;
  const int ch = blockIdx.x / strips;
  const int y = (blockIdx.x - ch * strips) * ROWS + w;
  const size_t off = ch * (size_t)H * M + (size_t)min(y, H - 1) * M;
  float2* tws = sm + ROWS * WR::BUF;
  stage_row_twiddles<M>(tws, twW);
  griddep_wait();
  if (SPEC && y < H) WR::stage_row(spec + off, sm + w * WR::BUF, lane);
  cp_async_wait_all();
  __syncthreads();
  if (y >= H) return;  // warp-uniform; no CTA barrier below
  WR::template inverse_row_to_global<EPI, SPEC>(spec + off, reinterpret_cast<float2*>(u), off, epi, sm + w * WR::BUF,
                                                lane, TwRef{tws, tws + M});
}

// Reverse-mode row pass of step n (the adjoint of Algorithm 1's iteration; see the generic
// row_adjoint_kernel for the derivation): warp w inverse-transforms strip row w of r = A^-1
// gbar (rows y0-1 .. y0+ROWS), then output warp o = w-1 forms, per pixel pair,
//   fbar += r,  gbar' = lambda/2 sum_* grad_*^T [ g''(grad_* u^n) * grad_* r ]
// (g'' of Appendix B; u^n read from global memory), and forward-transforms gbar' for the
// next step's column pass unless this is the last step (then gbar' goes to gu0 or fbar).
template <int PEN>
__device__ __forceinline__ float g2_pen(float x, const MuParams& mp) {
  const float x2 = x * x;
  if constexpr (PEN == 1) {
    return fmaf(-2.0f * sfu_exp2(-mp.wbeta * x2), fmaf(-2.0f * mp.winv2g2, x2, 1.0f), mp.c);
  } else {
    const float w = sfu_exp2((mp.a - 1.0f) * sfu_log2(x2 + mp.eps));
    return fmaf(-mp.p * w, fmaf(mp.p - 1.0f, x2, mp.eps), mp.c);
  }
}

template <int L, int ROWS, int PEN, int MINB>
__global__ void __launch_bounds__((ROWS + 2) * 32, MINB)
row_warp_adj_kernel(int H, const float2* __restrict__ twW, MuParams mp, const float2* __restrict__ spec_in,
                    const float* __restrict__ u_n, float* __restrict__ fbar, int fbar_first, float* __restrict__ gu0,
                    int last, float2* __restrict__ spec_out) {
  griddep_launch();
  griddep_wait();
  using WR = WarpRow<L>;
  constexpr int M = WR::M;
  extern __shared__ float2 sm[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int strips = (H + ROWS - 1) / ROWS;
  const int ch = blockIdx.x / strips;
  const int y0 = (blockIdx.x - ch * strips) * ROWS;
  const int nout = min(ROWS, H - y0);
  const size_t plane = (size_t)H * M;
  float2* buf = sm + w * WR::BUF;
  float2* tws = sm + (ROWS + 2) * WR::BUF;
  const TwRef tw{tws, tws + M};
  stage_row_twiddles<M>(tws, twW);
  cp_async_wait_all();
  __syncthreads();
  if (w < nout + 2)
    WR::template inverse_row_to_buf<false>(spec_in + ch * plane + (size_t)wrap_row(y0 - 1 + w, H) * M, buf, lane,
                                           tw);
  __syncthreads();
  const int o = w - 1;
  const bool out_live = o >= 0 && o < nout;
  float2 v[L];
  if (out_live) {
    const int y = y0 + o;
    const float2* uc = reinterpret_cast<const float2*>(u_n) + ch * plane;
    const float2* urow = uc + (size_t)y * M;
    const float2* uup = uc + (size_t)wrap_row(y - 1, H) * M;
    const float2* udn = uc + (size_t)wrap_row(y + 1, H) * M;
    const float2* rup = sm + (w - 1) * WR::BUF;
    const float2* rdn = sm + (w + 1) * WR::BUF;
    float2* fb = reinterpret_cast<float2*>(fbar) + ch * plane + (size_t)y * M;
    float2* g0 = gu0 != nullptr ? reinterpret_cast<float2*>(gu0) + ch * plane + (size_t)y * M : nullptr;
#pragma unroll
    for (int n2 = 0; n2 < L; ++n2) {
      const int m = lane + 32 * n2;
      const int ml = m == 0 ? M - 1 : m - 1, mr = m == M - 1 ? 0 : m + 1;
      const float2 rc = buf[m];
      const float rl = buf[ml].y, rrt = buf[mr].x;
      const float2 ru = rup[m], rd = rdn[m];
      const float2 u0c = urow[m];
      const float ul = urow[ml].y, ur = urow[mr].x;
      const float2 uu = uup[m], ud = udn[m];
      const float qx_l = g2_pen<PEN>(u0c.x - ul, mp) * (rc.x - rl);
      const float qx_c = g2_pen<PEN>(u0c.y - u0c.x, mp) * (rc.y - rc.x);
      const float qx_r = g2_pen<PEN>(ur - u0c.y, mp) * (rrt - rc.y);
      const float qy0u = g2_pen<PEN>(u0c.x - uu.x, mp) * (rc.x - ru.x);
      const float qy0d = g2_pen<PEN>(ud.x - u0c.x, mp) * (rd.x - rc.x);
      const float qy1u = g2_pen<PEN>(u0c.y - uu.y, mp) * (rc.y - ru.y);
      const float qy1d = g2_pen<PEN>(ud.y - u0c.y, mp) * (rd.y - rc.y);
      const float2 gb = c2(mp.half_lambda * ((qx_l - qx_c) + (qy0u - qy0d)),
                           mp.half_lambda * ((qx_c - qx_r) + (qy1u - qy1d)));
      float2 acc = fbar_first ? c2(0.0f, 0.0f) : fb[m];
      acc.x += rc.x;
      acc.y += rc.y;
      if (last && g0 == nullptr) {
        acc.x += gb.x;
        acc.y += gb.y;
      }
      fb[m] = acc;
      if (last && g0 != nullptr) g0[m] = gb;
      v[n2] = gb;
    }
  }
  if (last) return;  // kernel-uniform
  __syncthreads();   // every warp has read the r rows; buffer w becomes warp w's scratch
  if (out_live) WR::forward_row_to_global(v, spec_out + ch * plane + (size_t)(y0 + o) * M, buf, lane, tw);
}

// ---------------------------------------------------------------- two warps per row
//
// Rows of M = 64 L complex points (W = 128 L; W = 3840: L = 30) are transformed by a warp
// pair, so that a lane holds L values, as in the one-warp transform of a row half as long.
// Lane g = lane + 32 h of the pair (h: the pair's warp) holds x[g + 64 n2], n2 < L, runs the
// L-point DFT over its registers and multiplies by w_M^{g k2}; the pair transposes through
// the row's buffer (line stride 65, conflict free); lane k2 < L of warp h then runs the
// 32-point DFT Z_h of the stride-2 subsequence y[h + 2 b] of the 64 values of index k2, and
// one radix-2 step joins the halves of the 64-point DFT: Y[k + 32 c] = Z_0[k] + (-1)^c
// w_64^k Z_1[k], warp h forming c = h after the two warps swap their Z through the buffer.
// X[k2 + L k1] lands in register k1 - 32 h of lane k2 of warp h.  The pair synchronizes with
// its own named barrier (bar.sync 1 + pair, 64 threads), three times per transform.  The ids
// are immediates (one switch case per pair of the CTA) so that a CTA reserves only NP + 1
// hardware barriers; a register id would reserve all 16.
#define ILS_PAIR_BAR(k) \
  case k - 1:           \
    if constexpr (NP >= k) asm volatile("bar.sync " #k ", 64;" ::: "memory"); \
    break;
template <int L, int NP>
struct PairRow {
  static constexpr int M = 64 * L;
  static constexpr int STRIDE = 65;  // complex per transposed line
  static constexpr int BUF = (L * STRIDE > M ? L * STRIDE : M);
  static_assert(L <= 32 && L % 2 == 0, "one 32-point transform per lane; 16-byte row copies");
  static_assert(2 * 32 * L <= BUF, "the Z exchange fits the row buffer");

  static_assert(NP >= 1 && NP <= 15, "one named barrier per pair (ids 1..15)");
  // the pair barrier of pair p < NP
  __device__ __forceinline__ static void bar(int p) {
    switch (p) {
      ILS_PAIR_BAR(1) ILS_PAIR_BAR(2) ILS_PAIR_BAR(3) ILS_PAIR_BAR(4) ILS_PAIR_BAR(5)
      ILS_PAIR_BAR(6) ILS_PAIR_BAR(7) ILS_PAIR_BAR(8) ILS_PAIR_BAR(9) ILS_PAIR_BAR(10)
      ILS_PAIR_BAR(11) ILS_PAIR_BAR(12) ILS_PAIR_BAR(13) ILS_PAIR_BAR(14) ILS_PAIR_BAR(15)
      default: break;
    }
  }

  // v: lane g holds x[g + 64 n2]; out[k] (lane k2 < L of warp h): X[k2 + L (k + 32 h)].
  // buf: the pair's row buffer, free on entry; on return lane k2 of warp h may write the slots
  // k2 + L (k + 32 h) (its outputs' natural-order slots), the rest only after a pair barrier.
  template <bool INV>
  __device__ __forceinline__ static void fft(float2 (&v)[L], float2 (&out)[32], float2* buf, int g, int h, int lane,
                                             int pr, const TwRef& tw) {
    dft_reg<L, INV>(v);
#pragma unroll
    for (int k2 = 1; k2 < L; ++k2) {
      float2 w = tw.ft[64 * k2 + g];  // w_M^{g k2}
      if (INV) w.y = -w.y;
      v[k2] = cmul(v[k2], w);
    }
#pragma unroll
    for (int k2 = 0; k2 < L; ++k2) buf[k2 * STRIDE + g] = v[k2];
    bar(pr);
    const bool act = lane < L;  // lane = k2
    if (act) {
#pragma unroll
      for (int b = 0; b < 32; ++b) out[b] = buf[lane * STRIDE + h + 2 * b];
      dft_reg<32, INV>(out);
      if (h == 1) {
        constexpr Roots<64> w64{};
#pragma unroll
        for (int k = 1; k < 32; ++k) out[k] = twiddle_const<64, INV>(out[k], k, w64);
      }
    }
    bar(pr);  // every lane has read its line
    // Z_h goes to the other warp's output region (natural-order slots k2 + L (k + 32 (1 - h))),
    // so that after the barrier each lane reads, and its caller overwrites, only its own
    // warp's region: no barrier is needed before the outputs are stored.
    if (act) {
      float2* other = buf + (1 - h) * (32 * L);
#pragma unroll
      for (int k = 0; k < 32; ++k) other[k * L + lane] = out[k];
    }
    bar(pr);
    if (act) {
      const float2* mine = buf + h * (32 * L);
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        const float2 z = mine[k * L + lane];
        out[k] = h == 0 ? cadd(out[k], z) : csub(z, out[k]);
      }
    }
  }

  // 16-byte asynchronous copy of the packed spectrum row X into buf (the caller waits).
  __device__ __forceinline__ static void stage_row(const float2* __restrict__ X, float2* buf, int g) {
#pragma unroll
    for (int q = 0; q < L / 2; ++q) cp_async16(buf + 2 * (g + 64 * q), X + 2 * (g + 64 * q));
  }

  // Hermitian unpacking of the packed half spectrum for the inverse real transform (the
  // formula of WarpRow::load_c2r), v[n2] = Z[g + 64 n2]; X global, or staged in buf (then the
  // pair has read buf on return).
  template <bool STAGED>
  __device__ __forceinline__ static void load_c2r(const float2* __restrict__ X, float2 (&v)[L], const float2* buf,
                                                  int g, int pr, const TwRef& tw) {
    const float2* src = STAGED ? buf : X;
#pragma unroll
    for (int n2 = 0; n2 < L; ++n2) {
      const int k = g + 64 * n2;
      if (k == 0) {
        const float2 x = src[0];
        v[n2] = c2(x.x + x.y, x.x - x.y);
      } else {
        const float2 a = src[k], b = cconj(src[M - k]);
        const float2 s = cadd(a, b), d = csub(a, b);
        const float2 t = cmul(cconj(tw.rt[k]), d);
        v[n2] = c2(s.x - t.y, s.y + t.x);
      }
    }
    if (STAGED) bar(pr);
  }

  // Inverse real transform of X into buf in natural order (pairs of pixels, unnormalized);
  // the caller synchronizes before other warps read buf.
  __device__ __forceinline__ static void inverse_row_to_buf(const float2* __restrict__ X, float2* buf, int g, int h,
                                                            int lane, int pr, const TwRef& tw) {
    float2 v[L];
    load_c2r<false>(X, v, buf, g, pr, tw);
    float2 out[32];
    fft<true>(v, out, buf, g, h, lane, pr, tw);
    if (lane < L) {
#pragma unroll
      for (int k = 0; k < 32; ++k) buf[lane + L * (k + 32 * h)] = out[k];
    }
  }

  // Inverse real transform of X (global, or staged in buf) straight to the output through
  // the epilogue (pair index rowoff + m of the output image).
  template <int EPI, bool STAGED>
  __device__ __forceinline__ static void inverse_row_to_global(const float2* __restrict__ X, float2* out,
                                                               size_t rowoff, const Epilogue& epi, float2* buf, int g,
                                                               int h, int lane, int pr, const TwRef& tw) {
    float2 v[L];
    load_c2r<STAGED>(X, v, buf, g, pr, tw);
    float2 res[32];
    fft<true>(v, res, buf, g, h, lane, pr, tw);
    float dm = 0.0f;
    if (lane < L) {
#pragma unroll
      for (int k = 0; k < 32; ++k)
        dm = fmaxf(dm, epi.template store<EPI>(out, rowoff + lane + L * (k + 32 * h), res[k]));
    }
    epi.template finish<EPI>(dm);
  }

  // Forward real transform of r (lane g holds the r-pairs m = g + 64 n2) to the packed half
  // spectrum in dst; buf must be free for the pair (no other reader left).
  __device__ __forceinline__ static void forward_row_to_global(float2 (&v)[L], float2* dst, float2* buf, int g, int h,
                                                               int lane, int pr, const TwRef& tw) {
    float2 out[32];
    fft<false>(v, out, buf, g, h, lane, pr, tw);
    if (lane < L) {
#pragma unroll
      for (int k = 0; k < 32; ++k) buf[lane + L * (k + 32 * h)] = out[k];
    }
    bar(pr);
    // buf holds Z = FFT_M(r[2m] + i r[2m+1]): the packed half spectrum, pairs (k, M-k)
#pragma unroll
    for (int q = 0; q < (M / 2 + 1 + 63) / 64; ++q) {
      const int k = g + 64 * q;
      if (k > M / 2) continue;
      if (k == 0) {
        const float2 z = buf[0];
        dst[0] = c2(z.x + z.y, z.x - z.y);
      } else {
        const float2 a = buf[k], b = buf[M - k];
        const float2 fa = cscale(cadd(a, cconj(b)), 0.5f), fo = cscale(csub(a, cconj(b)), 0.5f);
        dst[k] = cadd(fa, cmul(tw.rt[k], c2(fo.y, -fo.x)));
        if (M - k != k) {
          const float2 fb = cscale(cadd(b, cconj(a)), 0.5f), fq = cscale(csub(b, cconj(a)), 0.5f);
          dst[M - k] = cadd(fb, cmul(tw.rt[M - k], c2(fq.y, -fq.x)));
        }
      }
    }
  }
};

// Fused row pass with a warp pair per strip row: CTA = ROWS + 2 pairs over rows y0-1 ..
// y0+ROWS (periodic); pair p holds strip row p in buffer p.  FIRST: u^0 rows are copied from
// u0 (or f); otherwise rebuilt by the inverse transform of spec_in.  Pair o+1 then forms r of
// output row o with the per-pair stencil of row_warp_fwd_kernel (mu of the pair's three x
// gradients and four y gradients; the x gradient left of a pair is the left lane's right
// one, lane 0 evaluating its own) and forward-transforms it.
template <int L, int ROWS, bool FIRST, int PEN, int MINB>
__global__ void __launch_bounds__((ROWS + 2) * 64, MINB)
row_pair_fwd_kernel(int H, const float2* __restrict__ twW, MuParams mp, const float* __restrict__ f,
                    const float* __restrict__ u0, const float2* __restrict__ spec_in, float2* __restrict__ spec_out,
                    float* __restrict__ u_ckpt) {
  griddep_launch();
  using PR = PairRow<L, ROWS + 2>;
  constexpr int M = PR::M;
  extern __shared__ float2 sm[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, p = w >> 1, h = w & 1, g = lane + 32 * h;
  const int strips = (H + ROWS - 1) / ROWS;
  const int ch = blockIdx.x / strips;
  const int y0 = (blockIdx.x - ch * strips) * ROWS;
  const int nout = min(ROWS, H - y0);
  const size_t plane = (size_t)H * M;
  float2* buf = sm + p * PR::BUF;
  auto U = [&](int row, int m) -> float2 { return sm[row * PR::BUF + m]; };
  const int o = p - 1;  // output row of this pair
  const bool out_live = o >= 0 && o < nout;
  const bool f_is_u = FIRST && (u0 == nullptr || u0 == f);
  const size_t orow = ch * plane + (size_t)(y0 + max(o, 0)) * M;
  float2* tws = sm + (ROWS + 2) * PR::BUF;
  const TwRef tw{tws, tws + M};
  stage_row_twiddles<M>(tws, twW);  // constant tables: before the wait on the previous grid
  griddep_wait();
  const int yy = wrap_row(y0 - 1 + p, H);
  if (FIRST && p < nout + 2) {
    const float2* src = reinterpret_cast<const float2*>(u0 != nullptr ? u0 : f) + ch * plane + (size_t)yy * M;
    if ((reinterpret_cast<size_t>(src) & 15) == 0) {
      PR::stage_row(src, buf, g);
    } else {
#pragma unroll
      for (int n2 = 0; n2 < L; ++n2) buf[g + 64 * n2] = src[g + 64 * n2];
    }
  }
  cp_async_wait_all();
  __syncthreads();
  if (!FIRST && p < nout + 2) PR::inverse_row_to_buf(spec_in + ch * plane + (size_t)yy * M, buf, g, h, lane, p, tw);
  __syncthreads();
  float2 v[L];
  if (mp.half_lambda == 0.0f) {  // lambda = 0 (or a plain row FFT): r = f
    if (out_live) {
      const float2* fr = reinterpret_cast<const float2*>(f) + orow;
#pragma unroll
      for (int n2 = 0; n2 < L; ++n2) {
        const int m = g + 64 * n2;
        v[n2] = fr[m];
        if (u_ckpt != nullptr) reinterpret_cast<float2*>(u_ckpt)[orow + m] = U(p, m);
      }
      PR::bar(p);  // both warps have read their row before the transform writes buf
      PR::forward_row_to_global(v, spec_out + orow, buf, g, h, lane, p, tw);
    }
    return;
  }
  if (out_live) {
    const float2* fr = reinterpret_cast<const float2*>(f) + orow;
#pragma unroll
    for (int n2 = 0; n2 < L; ++n2) {
      const int m = g + 64 * n2;
      const float2 c = U(p, m);
      const float ur = U(p, m == M - 1 ? 0 : m + 1).x;
      const float2 up = U(p - 1, m);
      const float2 dn = U(p + 1, m);
      const float2 fv = f_is_u ? c : fr[m];
      const float mx_c = mu_pen<PEN>(c.y - c.x, mp);
      const float mx_r = mu_pen<PEN>(ur - c.y, mp);
      float mx_l = __shfl_up_sync(kFull, mx_r, 1);
      if (lane == 0) mx_l = mu_pen<PEN>(c.x - U(p, m == 0 ? M - 1 : m - 1).y, mp);
      const float my0u = mu_pen<PEN>(c.x - up.x, mp);
      const float my0d = mu_pen<PEN>(dn.x - c.x, mp);
      const float my1u = mu_pen<PEN>(c.y - up.y, mp);
      const float my1d = mu_pen<PEN>(dn.y - c.y, mp);
      v[n2] = c2(fmaf(mp.half_lambda, (mx_l - mx_c) + (my0u - my0d), fv.x),
                 fmaf(mp.half_lambda, (mx_c - mx_r) + (my1u - my1d), fv.y));
      if (u_ckpt != nullptr) reinterpret_cast<float2*>(u_ckpt)[orow + m] = c;
    }
  }
  __syncthreads();  // every pair has read the strip rows: buffer p becomes pair p's scratch
  if (out_live) PR::forward_row_to_global(v, spec_out + orow, buf, g, h, lane, p, tw);
}

// Final inverse row pass with a warp pair per row, ROWS rows per CTA; EPI: the epilogue mode.
template <int L, int ROWS, int EPI, bool SPEC>
__global__ void __launch_bounds__(ROWS * 64)
row_pair_inv_kernel(int H, const float2* __restrict__ twW, const float2* __restrict__ spec, float* __restrict__ u,
                    Epilogue epi) {
  griddep_launch();
  using PR = PairRow<L, ROWS>;
  constexpr int M = PR::M;
  extern __shared__ float2 sm[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, p = w >> 1, h = w & 1, g = lane + 32 * h;
  const int strips = (H + ROWS - 1) / ROWS;
  const int ch = blockIdx.x / strips;
  const int y = (blockIdx.x - ch * strips) * ROWS + p;
  const size_t off = ch * (size_t)H * M + (size_t)min(y, H - 1) * M;
  float2* tws = sm + ROWS * PR::BUF;
  stage_row_twiddles<M>(tws, twW);
  griddep_wait();
  if (SPEC && y < H) PR::stage_row(spec + off, sm + p * PR::BUF, g);
  cp_async_wait_all();
  __syncthreads();
  if (y >= H) return;  // pair-uniform; no CTA barrier below
  PR::template inverse_row_to_global<EPI, SPEC>(spec + off, reinterpret_cast<float2*>(u), off, epi,
                                                sm + p * PR::BUF, g, h, lane, p, TwRef{tws, tws + M});
}

using FwdFn = void (*)(int, const float2*, MuParams, const float*, const float*, const float2*, float2*, float*);
using AdjFn = void (*)(int, const float2*, MuParams, const float2*, const float*, float*, int, float*, int, float2*);
using InvFn = void (*)(int, const float2*, const float2*, float*, Epilogue);

struct WarpRowEntry {
  int M, rows_fwd, rows_inv, buf, stage;
  int P;                     // warps per row: 1 (WarpRow) or 2 (PairRow)
  int rows_first;            // output rows per CTA of the first row pass (no inverse transforms)
  FwdFn first[kPenalties], later[kPenalties];  // per penalty (MuParams::pen)
  InvFn inv[kEpilogues];     // per epilogue mode
  AdjFn adj[2];              // per penalty with an adjoint (Eq. 7, Welsch)
};

// STAGE only where the staged rows still leave room for two CTAs per SM.  MINB: CTAs per SM
// the register allocation must allow (2 at 256 threads = 128 registers per thread).
// SPEC / SPEC_I: the row passes / the final inverse pass stage their spectrum rows in shared
// memory with 16-byte asynchronous copies (load_c2r from buf) instead of loading them directly.
template <int L, int RF, int RI, bool STAGE, bool SHARED, int MINB = ((RF + 2) * 32 <= 256 ? 2 : 1), bool SPEC = false,
          bool SPEC_I = SPEC>
constexpr WarpRowEntry warp_entry() {
  static_assert(SHARED || !STAGE, "f staging is part of the shared-mu stencil");
  return WarpRowEntry{32 * L,
                      RF,
                      RI,
                      WarpRow<L>::BUF,
                      STAGE ? RF * 32 * L : 0,
                      1,
                      RF,
                      {row_warp_fwd_kernel<L, RF, true, STAGE, SHARED, 0, MINB, SPEC>,
                       row_warp_fwd_kernel<L, RF, true, STAGE, SHARED, 1, MINB, SPEC>,
                       row_warp_fwd_kernel<L, RF, true, STAGE, SHARED, 2, MINB, SPEC>},
                      {row_warp_fwd_kernel<L, RF, false, STAGE, SHARED, 0, MINB, SPEC>,
                       row_warp_fwd_kernel<L, RF, false, STAGE, SHARED, 1, MINB, SPEC>,
                       row_warp_fwd_kernel<L, RF, false, STAGE, SHARED, 2, MINB, SPEC>},
                      {row_warp_inv_kernel<L, RI, 0, SPEC_I>, row_warp_inv_kernel<L, RI, 1, SPEC_I>,
                       row_warp_inv_kernel<L, RI, 2, SPEC_I>, row_warp_inv_kernel<L, RI, 3, SPEC_I>,
                       row_warp_inv_kernel<L, RI, 4, SPEC_I>, row_warp_inv_kernel<L, RI, 5, SPEC_I>},
                      {row_warp_adj_kernel<L, RF, 0, MINB>, row_warp_adj_kernel<L, RF, 1, MINB>}};
}

// Warp-pair rows (M = 64 L): RF output rows per CTA of the later row passes ((RF + 2) pairs,
// MINB CTAs per SM), RF1 (MINB1) in the first row pass, whose strips only copy their rows (no
// repeated inverse transforms of halo rows, so short strips at more CTAs per SM win there), RI
// rows per final-inverse CTA (SPEC_I: staged spectrum rows); no adjoint kernel.
template <int L, int RF1, int MINB1, int RF, int MINB, int RI, bool SPEC_I>
constexpr WarpRowEntry pair_entry() {
  return WarpRowEntry{64 * L,
                      RF,
                      RI,
                      PairRow<L, 1>::BUF,
                      0,
                      2,
                      RF1,
                      {row_pair_fwd_kernel<L, RF1, true, 0, MINB1>, row_pair_fwd_kernel<L, RF1, true, 1, MINB1>,
                       row_pair_fwd_kernel<L, RF1, true, 2, MINB1>},
                      {row_pair_fwd_kernel<L, RF, false, 0, MINB>, row_pair_fwd_kernel<L, RF, false, 1, MINB>,
                       row_pair_fwd_kernel<L, RF, false, 2, MINB>},
                      {row_pair_inv_kernel<L, RI, 0, SPEC_I>, row_pair_inv_kernel<L, RI, 1, SPEC_I>,
                       row_pair_inv_kernel<L, RI, 2, SPEC_I>, row_pair_inv_kernel<L, RI, 3, SPEC_I>,
                       row_pair_inv_kernel<L, RI, 4, SPEC_I>, row_pair_inv_kernel<L, RI, 5, SPEC_I>},
                      {nullptr, nullptr}};
}

// The first entry of a length is its default; the others are autotune alternatives.  Every
// CTA also holds its 2M-entry twiddle table (16 B per complex point of a row), which is what
// limits the 1920-wide rows to the per-pair stencil without f staging at two CTAs per SM.
const WarpRowEntry kWarpRows[] = {
    warp_entry<4, 6, 8, true, true, 3>(),    // W = 256: 8-warp CTAs, three per SM (80 registers)
    warp_entry<8, 14, 16, true, true>(),     // W = 512
    warp_entry<10, 14, 16, true, true>(),    // W = 640
    warp_entry<20, 6, 8, true, true>(),      // W = 1280
    warp_entry<30, 6, 8, false, false, 2, false, true>(),  // W = 1920: per-pair stencil, inverse pass staged
    warp_entry<32, 6, 8, false, true>(),     // W = 2048
    warp_entry<30, 6, 8, false, false, 2, true>(),   // W = 1920, row passes staged too
    warp_entry<30, 14, 8, false, false, 1, false, true>(),  // W = 1920, taller strips (16-warp CTAs)
    warp_entry<30, 6, 6, false, false, 2, false, true>(),   // W = 1920, 6-row inverse CTAs (3 per SM)
    warp_entry<30, 6, 8, false, true, 2, false, true>(),    // W = 1920, shared-mu stencil
    warp_entry<20, 6, 8, false, false>(),    // W = 1280, per-pair stencil
    warp_entry<32, 6, 8, false, false>(),    // W = 2048, per-pair stencil
    warp_entry<4, 14, 16, true, true>(),     // W = 256, 16-warp CTAs, one per SM (89 registers)
    pair_entry<30, 3, 2, 6, 1, 4, true>(),   // W = 3840: first pass 10-warp CTAs two per SM, later 16-warp
};

}  // namespace

int warp_row_variants(int M, int* idx, int max) {
  int n = 0;
  for (int i = 0; i < (int)(sizeof(kWarpRows) / sizeof(kWarpRows[0])) && n < max; ++i)
    if (kWarpRows[i].M == M) idx[n++] = i;
  return n;
}

bool warp_row_has_adjoint(int idx) { return kWarpRows[idx].adj[0] != nullptr; }

cudaError_t warp_set_attributes() {
  cudaError_t e;
  for (const WarpRowEntry& r : kWarpRows) {
    const int sf = ((r.rows_fwd + 2) * r.buf + r.stage + 2 * r.M) * (int)sizeof(float2);
    const int s1 = ((r.rows_first + 2) * r.buf + r.stage + 2 * r.M) * (int)sizeof(float2);
    const int si = (r.rows_inv * r.buf + 2 * r.M) * (int)sizeof(float2);
    for (int pen = 0; pen < kPenalties; ++pen) {
      if ((e = cudaFuncSetAttribute(r.first[pen], cudaFuncAttributeMaxDynamicSharedMemorySize, s1))) return e;
      if ((e = cudaFuncSetAttribute(r.later[pen], cudaFuncAttributeMaxDynamicSharedMemorySize, sf))) return e;
    }
    for (int m = 0; m < kEpilogues; ++m)
      if ((e = cudaFuncSetAttribute(r.inv[m], cudaFuncAttributeMaxDynamicSharedMemorySize, si))) return e;
    const int sa = ((r.rows_fwd + 2) * r.buf + 2 * r.M) * (int)sizeof(float2);
    for (int pen = 0; pen < 2 && r.adj[0] != nullptr; ++pen)
      if ((e = cudaFuncSetAttribute(r.adj[pen], cudaFuncAttributeMaxDynamicSharedMemorySize, sa))) return e;
  }
  return cudaSuccess;
}

cudaError_t warp_row_forward(int idx, const ImageDesc& d, const Tables& t, const MuParams& mp, const float* f,
                             const float* u0, const float2* spec_in, float2* spec_out, float* u_ckpt,
                             cudaStream_t stream) {
  const WarpRowEntry& r = kWarpRows[idx];
  const int rows = spec_in == nullptr ? r.rows_first : r.rows_fwd;
  const int blocks = (d.H + rows - 1) / rows * d.C;
  const size_t smem = ((size_t)(rows + 2) * r.buf + r.stage + 2 * r.M) * sizeof(float2);
  const int pen = mp.pen;
  FwdFn fn = spec_in == nullptr ? r.first[pen] : r.later[pen];
  return launch_k(d.pdl, fn, blocks, (rows + 2) * 32 * r.P, smem, stream, d.H, t.twW, mp, f, u0, spec_in, spec_out,
                  u_ckpt);
}

cudaError_t warp_row_adjoint(int idx, const ImageDesc& d, const Tables& t, const MuParams& mp,
                             const float2* spec_in, const float* u_n, float* fbar, bool fbar_first, float* gu0,
                             bool last, float2* spec_out, cudaStream_t stream) {
  const WarpRowEntry& r = kWarpRows[idx];
  if ((mp.pen != 0 && mp.pen != 1) || r.adj[0] == nullptr) return cudaErrorInvalidValue;
  const int blocks = (d.H + r.rows_fwd - 1) / r.rows_fwd * d.C;
  const size_t smem = ((size_t)(r.rows_fwd + 2) * r.buf + 2 * r.M) * sizeof(float2);
  return launch_k(d.pdl, r.adj[mp.pen], blocks, (r.rows_fwd + 2) * 32, smem, stream, d.H, t.twW, mp, spec_in, u_n,
                  fbar, (int)fbar_first, gu0, (int)last, spec_out);
}

cudaError_t warp_row_inverse(int idx, const ImageDesc& d, const Tables& t, const float2* spec, float* u,
                             cudaStream_t stream, const Epilogue& epi) {
  const WarpRowEntry& r = kWarpRows[idx];
  const int blocks = (d.H + r.rows_inv - 1) / r.rows_inv * d.C;
  const size_t smem = ((size_t)r.rows_inv * r.buf + 2 * r.M) * sizeof(float2);
  return launch_k(d.pdl, r.inv[epi.mode], blocks, r.rows_inv * 32 * r.P, smem, stream, d.H, t.twW, spec, u, epi);
}

}  // namespace ils
