// Internal declarations shared by the libils.so translation units.
#pragma once
#include <cuda_runtime.h>

#include <utility>
#include <vector>

#include "ils_fft.cuh"

namespace ils {

// Parameters of Eq. 7 for one image.
struct MuParams {
  float c;       // c0 = p eps^(p/2-1)  (Eq. 11)
  float p;
  float eps;
  float a;       // p/2 - 1
  float half_lambda;
  // 0 = generalized Charbonnier (Eq. 2, Eq. 7), 1 = Welsch (Eq. 18, Eq. 19), 2 = half-quadratic
  // splitting with phi = |x| (Eq. 14: Q1 is a soft threshold at thr; half_lambda holds beta_n)
  int pen = 0;
  float wbeta = 0.0f;    // Welsch: log2(e) / (2 gamma^2)
  float winv2g2 = 0.0f;  // Welsch: 1 / (2 gamma^2)
  float thr = 0.0f;      // half-quadratic splitting: lambda / (2 beta_n)
};

// 2^x and log2(x) on the special-function unit (PTX ex2.approx / lg2.approx, flush to
// zero; relative error about 2^-22, far inside the smoothing's FP32 parity bar).
__device__ __forceinline__ float sfu_exp2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sfu_log2(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Eq. 7: mu = c g - p g (g^2 + eps)^(p/2 - 1); g^2 + eps >= eps > 0, so no denormal inputs.
__device__ __forceinline__ float mu_eq7(float g, const MuParams& mp) {
  const float t = fmaf(g, g, mp.eps);
  return g * fmaf(-mp.p, sfu_exp2(mp.a * sfu_log2(t)), mp.c);
}

// Eq. 19 (Welsch penalty): mu = c g - 2 g exp(-g^2 / (2 gamma^2)), c = 2 (Eq. 20).
__device__ __forceinline__ float mu_welsch(float g, const MuParams& mp) {
  return g * fmaf(-2.0f, sfu_exp2(-mp.wbeta * g * g), mp.c);
}
// Q1 of Eq. 14 for phi = |x|: argmin_mu beta (g - mu)^2 + lambda |mu| = soft threshold.
__device__ __forceinline__ float mu_hqs_l1(float g, const MuParams& mp) {
  const float a = fabsf(g) - mp.thr;
  return a > 0.0f ? copysignf(a, g) : 0.0f;
}
// mu of the penalty PEN (MuParams::pen); the kernels are instantiated per penalty.
template <int PEN>
__device__ __forceinline__ float mu_pen(float g, const MuParams& mp) {
  if constexpr (PEN == 0) return mu_eq7(g, mp);
  else if constexpr (PEN == 1) return mu_welsch(g, mp);
  else return mu_hqs_l1(g, mp);
}
constexpr int kPenalties = 3;

// Output stage of the final inverse row pass (u = the smoothed image, pairs of pixels):
//   mode 0: out = u;
//   mode 1: out = f + s (u - f) per channel (detail enhancement: s = 1 - k, k the boost);
//   mode 2: luminance-only colour (Sec. 3.4, option I): f is the luma Y of the 3-plane image
//           rgb and out_c = rgb_c + s (u - Y) for the three planes;
//   mode 3: pixel-interleaved output: channel c0 + i / plane2 of pair i goes to dst, whose
//           pixels hold C channels each (out is not written);
//   mode 4: log-luminance tone mapping (Sec. 4.2: smoothing on the logarithm of the
//           luminance): f is l = ln Y of the 3-plane image rgb, u the base layer b, and
//           out_c = rgb_c exp(a l + s b + o) for the three planes;
//   mode 5: out = u, and the largest iterate change max |u - prev| (prev = u^{N-1}) of the
//           pass is max-reduced into *dmax (the bits of a non-negative float; a NaN change
//           counts as +inf): the fallback test of the warm-started smoother.
// store<MODE> returns the pair's contribution to that maximum (0 for the other modes); a
// kernel keeps the running maximum per thread and calls finish<MODE> once at its end.
struct Epilogue {
  int mode = 0;
  float s = 1.0f;
  float a = 0.0f, o = 0.0f;  // mode 4
  const float* f = nullptr;
  const float* rgb = nullptr;
  float* dst = nullptr;      // mode 3
  int C = 1, c0 = 0;         // mode 3: channels per pixel of dst, channel of the first plane
  size_t plane2 = 0;         // modes 2-4: pixel pairs per plane (H W / 2)
  const float* prev = nullptr;  // mode 5
  unsigned int* dmax = nullptr;  // mode 5
  // MODE is the kernel's compile-time copy of `mode` (one instantiation per mode)
  template <int MODE>
  __device__ __forceinline__ float store(float2* out, size_t i, float2 u) const {
    if constexpr (MODE == 0) {
      out[i] = u;
    } else if constexpr (MODE == 5) {
      out[i] = u;
      const float2 q = reinterpret_cast<const float2*>(prev)[i];
      const float d = fmaxf(fabsf(u.x - q.x), fabsf(u.y - q.y));
      // fmaxf drops a NaN operand: a NaN in either pair member must still read as a change
      return (u.x - q.x == u.x - q.x && u.y - q.y == u.y - q.y) ? d : __int_as_float(0x7f800000);
    } else if constexpr (MODE == 3) {
      // 32-bit split of the pair index (the host limits interleaved images to < 2^32 pairs)
      const unsigned ii = (unsigned)i, p2 = (unsigned)plane2;
      const unsigned c = ii / p2, q = ii - c * p2;
      float* px = dst + (size_t)2 * q * C + c0 + c;
      px[0] = u.x;
      px[C] = u.y;
    } else {
      const float2 fv = reinterpret_cast<const float2*>(f)[i];
      if constexpr (MODE == 4) {
        const float gx = expf(fmaf(a, fv.x, fmaf(s, u.x, o))), gy = expf(fmaf(a, fv.y, fmaf(s, u.y, o)));
        const float2* src = reinterpret_cast<const float2*>(rgb);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float2 v = src[c * plane2 + i];
          out[c * plane2 + i] = make_float2(v.x * gx, v.y * gy);
        }
      } else {
        const float dx = s * (u.x - fv.x), dy = s * (u.y - fv.y);
        if constexpr (MODE == 1) {
          out[i] = make_float2(fv.x + dx, fv.y + dy);
        } else {
          const float2* src = reinterpret_cast<const float2*>(rgb);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float2 v = src[c * plane2 + i];
            out[c * plane2 + i] = make_float2(v.x + dx, v.y + dy);
          }
        }
      }
    }
    return 0.0f;
  }
  // mode 5: max-reduce this thread's running maximum into *dmax, one atomic per warp (over
  // the lanes that reach the call; non-negative floats order like their bit patterns)
  template <int MODE>
  __device__ __forceinline__ void finish(float dm) const {
    if constexpr (MODE == 5) {
      const unsigned m = __activemask();
      const unsigned v = __reduce_max_sync(m, __float_as_uint(dm));
      if ((int)(threadIdx.x & 31) == __ffs(m) - 1) atomicMax(dmax, v);
    }
  }
};
constexpr int kEpilogues = 6;

// Launch geometry picked by the host planner (validated before any launch).
struct Geometry {
  int rows_fwd;      // output rows per CTA in the fused row pass (reads rows_fwd + 2 rows)
  int threads_row, ept_row;
  int rows_inv;      // rows per CTA in the final inverse row pass
  int threads_inv, ept_inv;
  int cols;          // complex columns per CTA in the column pass
  int threads_col, ept_col;
  size_t smem_fwd, smem_inv, smem_col;  // dynamic shared memory bytes
  int warp_row;      // index of a warp-per-row kernel for M = W/2, or -1
  int warp_adj;      // the warp-per-row kernel of the adjoint's row pass, or -1
  int fixed_row;     // index of a compile-time row plan for M = W/2, or -1 (generic kernels)
  int fixed_col;     // index of a compile-time column plan for H, or -1
};

// Lanes that share one packed row of M complex points in the warp-per-row transforms: 32
// (one warp, M = 32 L), or 64 (a warp pair, M = 64 L) for rows longer than 1024 points.
__host__ __device__ constexpr int four_step_lanes(int M) { return M > 1024 ? 64 : 32; }

// Device tables for one (H, W, lambda, c).
struct Tables {
  // exp(-2 pi i t / W) for t < W, then the W/2 four-step twiddles of the warp-per-row
  // transforms, k2-major so that the lanes of a row read consecutive entries:
  // twW[W + S k2 + n1] = exp(-2 pi i n1 k2 / (W/2)) with S = four_step_lanes(W/2)
  // (row_twiddles), then stage tables (row_twiddle_count)
  float2* twW;
  float2* twH;   // exp(-2 pi i t / H) for t < H, then stage tables (col_twiddle_count)
  float* ax;     // M+1 entries: lambda c (1 - cos(2 pi k / W)),  k = 0..M
  float* by;     // H entries:   lambda c (1 - cos(2 pi l / H)),  l = 0..H-1
};

// The first W + W/2 entries of Tables::twW for row length W (host, double precision, rounded
// once), padded with zeros to row_twiddle_count(W) for build_row_twiddles.
std::vector<float2> row_twiddles(int W);

struct ImageDesc {
  int H, W, C;
  FftPlan planM;  // length W/2 (row FFT on packed complex rows)
  FftPlan planH;  // length H   (column FFT)
  // Launch with programmatic dependent launch: set for every launch of a call except the
  // first, i.e. when the previous work on the stream is this library's own kernel.
  bool pdl = false;
};

// Programmatic dependent launch, device side.  Every ILS kernel lets the next grid be
// scheduled as soon as all of its CTAs run (launch_dependents), and reads nothing that the
// previous grid writes before griddep_wait() (which returns once that grid has completed
// and its writes are visible; a no-op for a kernel launched without the attribute).
__device__ __forceinline__ void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Whether the kernels of one call are chained by programmatic dependent launch (ILS_PDL=1).
// Off by default: on GB300 it measured 1% slower for a 1080p RGB frame and 3.6% slower for
// 24 channels than plain stream order.
bool pdl_enabled();

// Kernel launch with the programmatic-stream-serialization attribute when `pdl`.
template <typename... KArgs, typename... Args>
cudaError_t launch_k(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                     Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

bool make_fft_plan(int n, FftPlan* out);
bool pick_geometry(int H, int W, Geometry* g);

// Launchers (asynchronous on `stream`); return the launch error.
cudaError_t launch_row_forward(const ImageDesc& d, const Geometry& g, const Tables& t, const MuParams& mp,
                               const float* f, const float* u0, const float2* spec_in, float2* spec_out,
                               float* u_ckpt, cudaStream_t stream);
cudaError_t launch_col_solve(const ImageDesc& d, const Geometry& g, const Tables& t, float2* spec,
                             cudaStream_t stream);
cudaError_t launch_row_inverse(const ImageDesc& d, const Geometry& g, const Tables& t, const float2* spec,
                               float* u, cudaStream_t stream, const Epilogue& epi = Epilogue());
cudaError_t launch_row_adjoint(const ImageDesc& d, const Geometry& g, const Tables& t, const MuParams& mp,
                               const float2* spec_in, const float* u_n, float* fbar, bool fbar_first, float* gu0,
                               bool last, float2* spec_out, cudaStream_t stream);
cudaError_t set_kernel_attributes();
void record_cuda_error(const char* where, cudaError_t e);  // text for ils_last_error()
// 32->32 channel conv3x3 on tcgen05 tensor cores (ils_cnn_tc.cu)
bool conv32_tc_available();
cudaError_t conv32_tc_set_attributes();
cudaError_t launch_conv32_tc(int B, int H, int W, const void* in, const void* wt, const float* bias, void* out,
                             const void* mask, int relu, int* error, cudaStream_t st);
// 3->32 channel conv3x3 on tcgen05: in is NHWC BF16 rows of 8 channels (3 values, then zeros),
// wt [32][32] BF16 with column tap * 3 + ci (k < 27)
// u0 = f + conv3x3_{32->3}(in) + bias on tcgen05 (the warm-start network's last layer)
cudaError_t launch_conv_last_tc(int B, int H, int W, const void* in, const void* wt, const float* bias, const float* f,
                                float* u0, int* error, cudaStream_t st);
cudaError_t launch_conv3_tc(int B, int H, int W, const void* in8, const void* wt, const float* bias, void* out,
                            const void* mask, int relu, int* error, cudaStream_t st);
// weight and bias gradients of a conv3x3 with ci_n, co_n <= 32 on tcgen05, accumulated into
// dw [co_n][kpad] (column (3 dy + dx) ci_n + ci) and db [co_n]; x and dy are NHWC BF16 rows of
// 32 channels, or of 8 (channels beyond ci_n / co_n zero) for a side with at most 8
// (x_ch, dy_ch: channels per NHWC row of x and dy, 8 or 32)
cudaError_t launch_wgrad_tc(int B, int H, int W, const void* x, int x_ch, int ci_n, const void* dy, int dy_ch, int co_n,
                            float* dw, int kpad, float* db, int* error, cudaStream_t st);
// warm-start network inference as two fused tcgen05 kernels (ils_cnn_fused.cu)
cudaError_t warm_fused_set_attributes();
cudaError_t launch_warm_fused(int B, int H, int W, const float* f, void* act, float* u0, const void* const* w,
                              const float* const* bias, int* error, cudaStream_t st);

// Compile-time specialised kernels (ils_kernels_fixed.cu).
int fixed_row_index(int M);
int fixed_col_index(int H);
int fixed_row_variants(int M, int* idx, int max);  // all entries for a length (first = default)
int fixed_col_variants(int H, int* idx, int max);
cudaError_t fixed_set_attributes();
cudaError_t fixed_row_forward(int idx, const ImageDesc& d, const Tables& t, const MuParams& mp, const float* f,
                              const float* u0, const float2* spec_in, float2* spec_out, float* u_ckpt,
                              cudaStream_t stream);
cudaError_t fixed_row_inverse(int idx, const ImageDesc& d, const Tables& t, const float2* spec, float* u,
                              cudaStream_t stream, const Epilogue& epi);
cudaError_t fixed_col_solve(int idx, const ImageDesc& d, const Tables& t, float2* spec, cudaStream_t stream);
// Tables::twH holds col_twiddle_count(H) entries: the H roots, then the stage twiddle tables
// of the compile-time column plans of H, gathered from the roots by build_col_twiddles.
size_t col_twiddle_count(int H);
cudaError_t build_col_twiddles(int H, float2* twH, cudaStream_t st);
// Tables::twW holds row_twiddle_count(W) entries: the W roots, the W/2 four-step entries
// (row_twiddles), then the stage twiddle tables of the compile-time row plans of W/2,
// gathered from the roots by build_row_twiddles.
size_t row_twiddle_count(int W);
cudaError_t build_row_twiddles(int W, float2* twW, cudaStream_t st);

// Warp-per-row kernels (ils_rows_warp.cu).
int warp_row_variants(int M, int* idx, int max);
// whether warp-per-row entry idx has an adjoint row kernel (the warp-pair entries have none)
bool warp_row_has_adjoint(int idx);
cudaError_t warp_set_attributes();
cudaError_t warp_row_forward(int idx, const ImageDesc& d, const Tables& t, const MuParams& mp, const float* f,
                             const float* u0, const float2* spec_in, float2* spec_out, float* u_ckpt,
                             cudaStream_t stream);
cudaError_t warp_row_adjoint(int idx, const ImageDesc& d, const Tables& t, const MuParams& mp,
                             const float2* spec_in, const float* u_n, float* fbar, bool fbar_first, float* gu0,
                             bool last, float2* spec_out, cudaStream_t stream);
cudaError_t warp_row_inverse(int idx, const ImageDesc& d, const Tables& t, const float2* spec, float* u,
                             cudaStream_t stream, const Epilogue& epi);

}  // namespace ils
