// ils_smooth_noalloc: the ILS iteration with its workspace in a fixed, file-scope
// device array instead of memory from cudaMalloc.
//
// Some callers cannot allocate device memory once they are running: a video
// pipeline that must hold its frame rate cannot afford cudaMalloc's implicit
// device synchronization and unbounded latency in the middle of a stream, and
// a plugin hosted inside another application may not own any allocation at
// all.  This entry point gives them the same smoothing with no allocation of
// any kind (no cudaMalloc/cudaFree, no host heap, no library allocator); the
// caller still provides the input and output buffers.
#include <cuda.h>  // CUcontext, CUresult: two driver calls resolved at run time
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/ils.h"
#include "ils_internal.h"

using namespace ils;

namespace {

constexpr int kSideMax = ILS_NOALLOC_MAX_SIDE;
constexpr size_t kElemsMax = ILS_NOALLOC_MAX_ELEMS;  // floats per image (C*H*W)
// table floats: twW (3*side + 2*kStageTw: W + W/2 complex and the row plans' stage tables) +
// twH (2*(side + kStageTw): H roots and the column plans' stage tables) + ax (side/2+1,
// padded) + by (side)
constexpr size_t kStageTw = 16384;  // complex; at least the stage-table part of every length
constexpr size_t kTwW = 3 * kSideMax + 2 * kStageTw;
constexpr size_t kTableFloats = kTwW + 2 * (kSideMax + kStageTw) + (kSideMax / 2 + 64) + kSideMax;
constexpr size_t kScratchFloats = 2 * kElemsMax + kTableFloats;

// Shared by every call on a device and kept until the process exits.
static __device__ __align__(256) float g_noalloc_scratch[kScratchFloats];

static_assert(kScratchFloats * sizeof(float) == ILS_NOALLOC_SCRATCH_BYTES, "the header states the array's size");

// A __device__ array has one instance per CUDA context, and its address is only valid in
// that context.  The address (and whether the kernels' shared-memory limits have been set,
// which is also per context) is therefore cached per context, keyed by the context's
// process-unique identifier: a context made current by a host application, or a primary
// context re-created after cudaDeviceReset, gets its own set-up.
struct CtxEntry {
  unsigned long long id;
  void* scratch;
};
constexpr int kMaxContexts = 64;
std::mutex g_mu;
CtxEntry g_ctx[kMaxContexts] = {};
int g_nctx = 0, g_next = 0;

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// The calling thread's current context identifier (driver calls resolved at run time; the
// library links only the CUDA runtime).
ils_status current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static const bool resolved = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(p);
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(p);
    return get_current != nullptr && get_id != nullptr;
  }();
  if (!resolved) return ILS_ERR_CUDA;
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS) return ILS_ERR_CUDA;
  if (ctx == nullptr) {
    // no context bound to this thread yet: a runtime call binds the device's primary context
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return ILS_ERR_CUDA;
    if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return ILS_ERR_CUDA;
  }
  return get_id(ctx, id) == CUDA_SUCCESS ? ILS_OK : ILS_ERR_CUDA;
}

// Device address of the scratch array in the current context; the first call in a context
// resolves it (and sets the kernels' shared-memory limits) with that context current.
ils_status scratch_for_current_context(float** out) {
  unsigned long long id = 0;
  ils_status s = current_context_id(&id);
  if (s != ILS_OK) return s;
  std::lock_guard<std::mutex> lock(g_mu);
  for (int i = 0; i < g_nctx; ++i) {
    if (g_ctx[i].id == id) {
      *out = static_cast<float*>(g_ctx[i].scratch);
      return ILS_OK;
    }
  }
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return ILS_ERR_CUDA;
  if (set_kernel_attributes() != cudaSuccess) return ILS_ERR_CUDA;
  // the oldest entry makes room when every slot is taken (its context may be gone)
  const int slot = g_nctx < kMaxContexts ? g_nctx++ : (g_next++ % kMaxContexts);
  g_ctx[slot] = CtxEntry{id, p};
  *out = static_cast<float*>(p);
  return ILS_OK;
}

// Twiddle and Eq. 9 denominator tables, computed on the device in double precision.
__global__ void noalloc_tables_kernel(int H, int W, double lc, float2* twW, float2* twH, float* ax, float* by) {
  const int M = W / 2;
  const int n = W > H ? W : H;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double s, c;
    if (i < W) {
      sincospi(-2.0 * (double)i / (double)W, &s, &c);
      twW[i] = make_float2((float)c, (float)s);
    }
    if (i < M) {  // the four-step entries (layout of Tables::twW): the same values as twW[2 n1 k2 mod W]
      const int S = four_step_lanes(M), k2 = i / S, n1 = i % S;
      sincospi(-2.0 * (double)((2 * n1 * k2) % W) / (double)W, &s, &c);
      twW[W + i] = make_float2((float)c, (float)s);
    }
    if (i < H) {
      sincospi(-2.0 * (double)i / (double)H, &s, &c);
      twH[i] = make_float2((float)c, (float)s);
      const double sh = sinpi((double)i / (double)H);
      by[i] = (float)(2.0 * lc * sh * sh);
    }
    if (i <= M) {
      const double sw = sinpi((double)i / (double)W);
      ax[i] = (float)(2.0 * lc * sw * sw);
    }
  }
}

bool smooth_235(int n) {
  if (n < 1) return false;
  for (int r : {2, 3, 5})
    while (n % r == 0) n /= r;
  return n == 1;
}

}  // namespace

extern "C" ils_status ils_smooth_noalloc(int H, int W, int C, float lambda, float p, float eps, int N,
                                         const float* f, float* u, void* stream) {
  if (f == nullptr || u == nullptr) return ILS_ERR_INVALID_ARG;
  if (C < 1 || N < 0 || !(lambda >= 0.0f) || !std::isfinite(lambda) || !(eps > 0.0f) || !std::isfinite(eps) ||
      !((p > 0.0f && p <= 1.0f) || p == 2.0f))
    return ILS_ERR_INVALID_ARG;
  if (H < 2 || W < 2 || H > kSideMax || W > kSideMax || (W & 1) || !smooth_235(H) || !smooth_235(W))
    return ILS_ERR_UNSUPPORTED_SIZE;
  const size_t elems = (size_t)C * (size_t)H * (size_t)W;
  if (elems > kElemsMax) return ILS_ERR_UNSUPPORTED_SIZE;  // beyond the fixed scratch array
  const size_t bytes = elems * sizeof(float);
  const uintptr_t a = reinterpret_cast<uintptr_t>(f), b = reinterpret_cast<uintptr_t>(u);
  if (a < b + bytes && b < a + bytes) return ILS_ERR_INVALID_ARG;

  ImageDesc d;
  d.H = H; d.W = W; d.C = C;
  Geometry g;
  if (!make_fft_plan(W / 2, &d.planM) || !make_fft_plan(H, &d.planH) || !pick_geometry(H, W, &g))
    return ILS_ERR_UNSUPPORTED_SIZE;

  float* base = nullptr;
  ils_status s = scratch_for_current_context(&base);
  if (s != ILS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (N == 0) {
    e = cudaMemcpyAsync(u, f, bytes, cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? ILS_OK : ILS_ERR_CUDA;
  }
  // scratch layout (floats): spectrum 0 | spectrum 1 | twW | twH | ax | by
  float2* spec[2] = {reinterpret_cast<float2*>(base), reinterpret_cast<float2*>(base + kElemsMax)};
  float* tab = base + 2 * kElemsMax;
  Tables t;
  t.twW = reinterpret_cast<float2*>(tab);
  t.twH = reinterpret_cast<float2*>(tab + kTwW);
  t.ax = tab + kTwW + 2 * (kSideMax + kStageTw);
  t.by = t.ax + (kSideMax / 2 + 64);
  if (col_twiddle_count(H) > (size_t)kSideMax + kStageTw || 2 * row_twiddle_count(W) > kTwW)
    return ILS_ERR_UNSUPPORTED_SIZE;

  const double c = (double)p * std::pow((double)eps, (double)p / 2.0 - 1.0);
  MuParams mp;
  mp.c = (float)c;
  mp.p = p;
  mp.eps = eps;
  mp.a = p / 2.0f - 1.0f;
  mp.half_lambda = 0.5f * lambda;

  noalloc_tables_kernel<<<(kSideMax + 255) / 256, 256, 0, st>>>(H, W, (double)lambda * c, t.twW, t.twH, t.ax, t.by);
  if ((e = cudaGetLastError())) return ILS_ERR_CUDA;
  if ((e = build_col_twiddles(H, t.twH, st)) || (e = build_row_twiddles(W, t.twW, st))) return ILS_ERR_CUDA;
  for (int it = 0; it < N; ++it) {
    float2* out = spec[it & 1];
    const float2* in = it == 0 ? nullptr : spec[(it - 1) & 1];
    d.pdl = it > 0 && pdl_enabled();  // after the table kernel: stream order; then chained (programmatic)
    if ((e = launch_row_forward(d, g, t, mp, f, nullptr, in, out, nullptr, st))) return ILS_ERR_CUDA;
    d.pdl = pdl_enabled();
    if ((e = launch_col_solve(d, g, t, out, st))) return ILS_ERR_CUDA;
  }
  if ((e = launch_row_inverse(d, g, t, spec[(N - 1) & 1], u, st))) return ILS_ERR_CUDA;
  return ILS_OK;
}
