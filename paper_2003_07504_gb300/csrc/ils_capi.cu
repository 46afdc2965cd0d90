// C ABI of libils.so (declared in include/ils.h): plans, validation, tables and
// the iteration driver of Algorithm 1.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ils.h"
#include "ils_internal.h"

using namespace ils;

namespace ils {
cudaError_t launch_gaussian_blur(const float* f, float* out, int H, int W, int C, float sigma, cudaStream_t st);
}

// What a launch sequence of a plan depends on besides the plan itself.
struct LaunchKey {
  const float* f;
  const float* u0;
  float* u;
  float* ckpt;
  ils::Epilogue epi;
  const float* f_host;  // host input copied to f, and u copied to u_host, per channel group
  float* u_host;
  bool operator==(const LaunchKey& o) const {
    return f == o.f && u0 == o.u0 && u == o.u && ckpt == o.ckpt && f_host == o.f_host && u_host == o.u_host &&
           epi.mode == o.epi.mode && epi.s == o.epi.s &&
           epi.a == o.epi.a && epi.o == o.epi.o && epi.f == o.epi.f && epi.rgb == o.epi.rgb && epi.dst == o.epi.dst &&
           epi.C == o.epi.C && epi.c0 == o.epi.c0 && epi.plane2 == o.epi.plane2 && epi.prev == o.epi.prev &&
           epi.dmax == o.epi.dmax;
  }
};
struct GraphEntry {
  LaunchKey key;
  cudaGraphExec_t exec;  // null: the capture failed (e.g. pageable host memory); launch directly
  unsigned long long last_use;
};
constexpr size_t kMaxGraphs = 8, kMaxSeen = 16;

struct ils_plan {
  int H, W, C, N;
  float lambda, p, eps, c;
  int device;
  ImageDesc desc;
  Geometry geo;
  Tables tab;
  MuParams mp;
  float2* spec[2];     // ping-pong row-spectrum workspaces, C*H*(W/2) complex each
  float* stage_f;      // device staging for ils_smooth_host
  float* stage_u;
  float* luma;         // luminance of ils_smooth_luma (H x W), allocated at its first call
  // plan-owned checkpoints (ils_set_checkpointing): while on, ils_smooth / ils_smooth_from store
  // u^0 .. u^{N-1} here, and ils_backward differentiates the last such call (its f, u0 kept)
  float* ckpt_own;
  const float* ckpt_f;
  const float* ckpt_u0;
  bool ckpt_valid;
  // half-quadratic splitting: per-iteration Eq. 14 parameters and denominator tables
  // (iteration n: ax at iter_tab + n (M + 1 + H), by right after it)
  std::vector<MuParams> mp_iter;
  float* iter_tab;
  // channels run on `nsplit` internal streams forked from and joined back to the caller's
  // stream, so that the small per-pass grids of a frame overlap each other's fill and drain
  int nsplit;
  std::vector<cudaStream_t> side;
  // [0] fork, [1 + s] join of side stream s, [1 + nsplit + s] its host input copied
  std::vector<cudaEvent_t> fork_join;
  // CUDA graphs of this plan's launch sequence, keyed by the call's pointers and output
  // stage (run_ils): a key seen twice is captured once and then replayed
  std::vector<GraphEntry> graphs;
  std::vector<LaunchKey> seen;
  cudaStream_t cap_stream;
  unsigned long long calls, captures, replays;
  // optional per-kernel event timing (ils_set_profiling)
  bool profiling;
  std::vector<cudaEvent_t> ev;  // one event before each launch plus one after the last
  std::vector<int> ev_kind;     // kind of the launch that starts at event i
  double prof_ms[ILS_KERNEL_KINDS];
  long long prof_launches[ILS_KERNEL_KINDS];
};

namespace {

// NVTX range over a scope (host side): a profiler attached to the process shows each
// call and each pass launch of Algorithm 1; without one the calls cost a pointer test.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

thread_local std::string g_last_error;

ils_status cuda_fail(cudaError_t e, const char* where) {
  g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
  return ILS_ERR_CUDA;
}

// Test hook: ILS_TEST_FAIL_ALLOC=k makes the k-th device allocation (1-based)
// of an ils_plan_create call report out-of-memory.
thread_local int g_alloc_count = 0;

ils_status dev_alloc(void** p, size_t bytes) {
  *p = nullptr;
  const char* env = std::getenv("ILS_TEST_FAIL_ALLOC");
  ++g_alloc_count;
  if (env != nullptr && std::atoi(env) == g_alloc_count) {
    g_last_error = "injected allocation failure";
    return ILS_ERR_OOM;
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    g_last_error = "cudaMalloc: out of memory";
    *p = nullptr;
    return ILS_ERR_OOM;
  }
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_fail(e, "cudaMalloc");
  }
  return ILS_OK;
}

bool smooth_235(int n) {
  if (n < 1) return false;
  for (int r : {2, 3, 5})
    while (n % r == 0) n /= r;
  return n == 1;
}

// [a, a + na) and [b, b + nb) intersect
bool overlaps2(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + nb && y < x + na;
}
bool overlaps(const void* a, const void* b, size_t bytes) { return overlaps2(a, bytes, b, bytes); }

void destroy_events(ils_plan* pl) {
  for (cudaEvent_t e : pl->ev) cudaEventDestroy(e);
  pl->ev.clear();
  pl->ev_kind.clear();
}

void free_plan_memory(ils_plan* pl) {
  destroy_events(pl);
  for (GraphEntry& g : pl->graphs) cudaGraphExecDestroy(g.exec);
  pl->graphs.clear();
  if (pl->cap_stream != nullptr) cudaStreamDestroy(pl->cap_stream);
  pl->cap_stream = nullptr;
  for (cudaStream_t x : pl->side) cudaStreamDestroy(x);
  for (cudaEvent_t x : pl->fork_join) cudaEventDestroy(x);
  pl->side.clear();
  pl->fork_join.clear();
  cudaFree(pl->spec[0]);
  cudaFree(pl->spec[1]);
  cudaFree(pl->stage_f);
  cudaFree(pl->stage_u);
  cudaFree(pl->luma);
  cudaFree(pl->ckpt_own);
  cudaFree(pl->iter_tab);
  cudaFree(pl->tab.twW);
  cudaFree(pl->tab.twH);
  cudaFree(pl->tab.ax);
  cudaFree(pl->tab.by);
}

// With profiling on, records an event before launch number `slot` of this call.
cudaError_t mark(ils_plan* pl, int slot, int kind, cudaStream_t st) {
  if (!pl->profiling) return cudaSuccess;
  pl->ev_kind[slot] = kind;
  return cudaEventRecord(pl->ev[slot], st);
}

// Y = 0.299 R + 0.587 G + 0.114 B (BT.601 luma) of a 3-plane image, n pixels per plane.
__global__ void luma_kernel(const float* __restrict__ rgb, float* __restrict__ y, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = fmaf(0.299f, rgb[i], fmaf(0.587f, rgb[n + i], 0.114f * rgb[2 * n + i]));
}

// l = ln max(Y, kLumaFloor) with Y the BT.601 luma of a 3-plane image (the log-luminance
// that Sec. 4.2 smooths for HDR tone mapping; the floor keeps l finite on black pixels).
constexpr float kLumaFloor = 1e-12f;
__global__ void log_luma_kernel(const float* __restrict__ rgb, float* __restrict__ l, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    l[i] = logf(fmaxf(fmaf(0.299f, rgb[i], fmaf(0.587f, rgb[n + i], 0.114f * rgb[2 * n + i])), kLumaFloor));
}

// Pixel-interleaved (H x W x C) to planar (C x H x W); one thread per pixel.
__global__ void hwc_to_planar_kernel(const float* __restrict__ src, float* __restrict__ dst, int C, size_t hw) {
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < hw; p += (size_t)gridDim.x * blockDim.x)
    for (int c = 0; c < C; ++c) dst[c * hw + p] = src[p * C + c];
}

// The output stage alone, with u = f (a plan with N = 0: u^0 = f is the result).
template <int MODE>
__global__ void epilogue_only_kernel(Epilogue epi, const float* __restrict__ f, float* out, size_t pairs) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < pairs; i += (size_t)gridDim.x * blockDim.x)
    epi.template store<MODE>(reinterpret_cast<float2*>(out), i, reinterpret_cast<const float2*>(f)[i]);
}

int grid_for(size_t n) { return (int)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, 4096)); }

// Parameters and tables of iteration `it` (the same for every iteration unless the plan is a
// half-quadratic-splitting one, whose weight beta_n changes).
const MuParams& iter_mp(const ils_plan* pl, int it) { return pl->mp_iter.empty() ? pl->mp : pl->mp_iter[it]; }
Tables iter_tab(const ils_plan* pl, int it) {
  Tables t = pl->tab;
  if (pl->iter_tab != nullptr) {
    t.ax = pl->iter_tab + (size_t)it * (pl->W / 2 + 1 + pl->H);
    t.by = t.ax + pl->W / 2 + 1;
  }
  return t;
}

// The 2N+1 launches of Algorithm 1 for channels [c0, c0 + cn) of the plan on `st` (pointers
// are those of channel 0; each channel's image, spectrum and checkpoint slices are disjoint).
// `slot` (profiling) counts the event marks between launches, or is null.
ils_status enqueue_ils(ils_plan* pl, int c0, int cn, const float* f, const float* u0, float* u, float* ckpt,
                       cudaStream_t st, const Epilogue& epi_in, int* slot) {
  const size_t hw = (size_t)pl->H * pl->W, n = (size_t)pl->C * hw, off = (size_t)c0 * hw;
  ImageDesc d = pl->desc;
  d.C = cn;
  Epilogue epi = epi_in;
  if (epi.mode == 1) epi.f += off;
  if (epi.mode == 3) epi.c0 += c0;
  if (epi.mode == 5) epi.prev += off;
  f += off;
  u += off;
  if (u0 != nullptr) u0 += off;
  float2* spec[2] = {pl->spec[0] + off / 2, pl->spec[1] + off / 2};
  cudaError_t e;
  auto mark_if = [&](int kind) -> cudaError_t { return slot ? mark(pl, (*slot)++, kind, st) : cudaSuccess; };
  // programmatic dependent launch between this call's own kernels (not after the caller's
  // work, and not when profiling events sit between the launches)
  const bool chain = slot == nullptr && pdl_enabled();
  for (int it = 0; it < pl->N; ++it) {
    float2* out = spec[it & 1];
    const float2* in = it == 0 ? nullptr : spec[(it - 1) & 1];
    float* ck = ckpt ? ckpt + (size_t)it * n + off : nullptr;
    if ((e = mark_if(it == 0 ? ILS_KERNEL_ROW_FIRST : ILS_KERNEL_ROW))) return cuda_fail(e, "event");
    d.pdl = chain && it > 0;
    const Tables tn = iter_tab(pl, it);
    {
      NvtxRange r(it == 0 ? "ils row pass n=0" : "ils row pass");
      if ((e = launch_row_forward(d, pl->geo, tn, iter_mp(pl, it), f, it == 0 ? u0 : nullptr, in, out, ck, st)))
        return cuda_fail(e, "row pass launch");
    }
    if ((e = mark_if(ILS_KERNEL_COLUMN))) return cuda_fail(e, "event");
    d.pdl = chain;
    NvtxRange rc("ils column pass");
    if ((e = launch_col_solve(d, pl->geo, tn, out, st))) return cuda_fail(e, "column pass launch");
  }
  if ((e = mark_if(ILS_KERNEL_ROW_INVERSE))) return cuda_fail(e, "event");
  d.pdl = chain;
  NvtxRange ri("ils final inverse row pass");
  if ((e = launch_row_inverse(d, pl->geo, pl->tab, spec[(pl->N - 1) & 1], u, st, epi)))
    return cuda_fail(e, "inverse row pass launch");
  return ILS_OK;
}

ils_status launch_all(ils_plan* pl, const LaunchKey& k, cudaStream_t st);

// Whether calls replay CUDA graphs of their launch sequence (ILS_GRAPHS=0 turns it off).
bool graphs_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("ILS_GRAPHS");
    return !(e != nullptr && e[0] == '0');
  }();
  return on;
}

// Captures the launch sequence for `key` on the plan's capture stream; null on any failure
// (the caller then launches directly).
cudaGraphExec_t capture(ils_plan* pl, const LaunchKey& key) {
  if (pl->cap_stream == nullptr && cudaStreamCreateWithFlags(&pl->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    pl->cap_stream = nullptr;
    return nullptr;
  }
  if (cudaStreamBeginCapture(pl->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return nullptr;
  const ils_status s = launch_all(pl, key, pl->cap_stream);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(pl->cap_stream, &g);
  cudaGraphExec_t exec = nullptr;
  if (s == ILS_OK && e == cudaSuccess && g != nullptr && cudaGraphInstantiate(&exec, g, 0) != cudaSuccess)
    exec = nullptr;
  if (g != nullptr) cudaGraphDestroy(g);
  cudaGetLastError();  // a failed capture leaves no sticky error; clear the last one
  return exec;
}

// Algorithm 1 for one call: replays the CUDA graph of this call's launch sequence when the
// same pointers and output stage were seen before (a video pipeline's steady state; measured
// at 1920 x 1080, N = 4: RGB 267 -> 258 us, gray 186 -> 166 us against stream launches),
// otherwise launches directly.  Not while profiling, for N = 0, or when the caller's stream
// is itself being captured.
ils_status run_ils(ils_plan* pl, const float* f, const float* u0, float* u, float* ckpt, cudaStream_t st,
                   const Epilogue& epi = Epilogue(), const float* f_host = nullptr, float* u_host = nullptr) {
  const LaunchKey key{f, u0, u, ckpt, epi, f_host, u_host};
  NvtxRange call("ils call");
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (pl->N == 0 || pl->profiling || !graphs_enabled() || cudaStreamIsCapturing(st, &cs) != cudaSuccess ||
      cs != cudaStreamCaptureStatusNone)
    return launch_all(pl, key, st);
  ++pl->calls;
  for (GraphEntry& g : pl->graphs) {
    if (g.key == key) {
      g.last_use = pl->calls;
      if (g.exec == nullptr) return launch_all(pl, key, st);
      ++pl->replays;
      const cudaError_t e = cudaGraphLaunch(g.exec, st);
      return e == cudaSuccess ? ILS_OK : cuda_fail(e, "cudaGraphLaunch");
    }
  }
  // a caller whose pointer sets rarely repeat (more sets in rotation than graphs kept) would
  // pay a capture per call: after 4 captures, capture again only if graphs are replayed
  // at least 4 times per capture
  if (pl->captures >= 4 && pl->replays < 4 * pl->captures) return launch_all(pl, key, st);
  bool seen = false;
  for (const LaunchKey& k : pl->seen) seen = seen || k == key;
  if (!seen) {
    if (pl->seen.size() == kMaxSeen) pl->seen.erase(pl->seen.begin());
    pl->seen.push_back(key);
    return launch_all(pl, key, st);
  }
  cudaGraphExec_t exec = capture(pl, key);
  ++pl->captures;
  if (pl->graphs.size() == kMaxGraphs) {  // evict the least recently used
    size_t lru = 0;
    for (size_t i = 1; i < pl->graphs.size(); ++i)
      if (pl->graphs[i].last_use < pl->graphs[lru].last_use) lru = i;
    if (pl->graphs[lru].exec != nullptr) cudaGraphExecDestroy(pl->graphs[lru].exec);
    pl->graphs.erase(pl->graphs.begin() + lru);
  }
  pl->graphs.push_back(GraphEntry{key, exec, pl->calls});
  if (exec == nullptr) return launch_all(pl, key, st);
  const cudaError_t e = cudaGraphLaunch(exec, st);
  return e == cudaSuccess ? ILS_OK : cuda_fail(e, "cudaGraphLaunch");
}

// Host copies of channels [c0, c0 + cn) for a host-buffer call (k.f_host / k.u_host).
cudaError_t host_in(ils_plan* pl, const LaunchKey& k, int c0, int cn, cudaStream_t st) {
  if (k.f_host == nullptr) return cudaSuccess;
  const size_t hw = (size_t)pl->H * pl->W;
  return cudaMemcpyAsync(const_cast<float*>(k.f) + c0 * hw, k.f_host + c0 * hw, cn * hw * sizeof(float),
                         cudaMemcpyHostToDevice, st);
}
cudaError_t host_out(ils_plan* pl, const LaunchKey& k, int c0, int cn, cudaStream_t st) {
  if (k.u_host == nullptr) return cudaSuccess;
  const size_t hw = (size_t)pl->H * pl->W;
  return cudaMemcpyAsync(k.u_host + c0 * hw, k.u + c0 * hw, cn * hw * sizeof(float), cudaMemcpyDeviceToHost, st);
}

// The launches of one call on `st` (2N + 1 kernels, or a copy for N = 0).  For host buffers
// each channel group's input copy, kernels and output copy run in order on its stream, so the
// copies of one group overlap the kernels of the others.
ils_status launch_all(ils_plan* pl, const LaunchKey& k, cudaStream_t st) {
  const float* f = k.f;
  const float* u0 = k.u0;
  float* u = k.u;
  float* ckpt = k.ckpt;
  const Epilogue& epi = k.epi;
  const size_t n = (size_t)pl->C * pl->H * pl->W;
  const size_t bytes = n * sizeof(float);
  cudaError_t e;
  if (pl->N == 0) {
    if ((e = host_in(pl, k, 0, pl->C, st))) return cuda_fail(e, "H2D copy");
    if (epi.mode == 3 || epi.mode == 4) {  // u = f through the output stage
      const size_t pairs = n / 2;
      if (epi.mode == 3) epilogue_only_kernel<3><<<grid_for(pairs), 256, 0, st>>>(epi, f, u, pairs);
      else epilogue_only_kernel<4><<<grid_for(pairs), 256, 0, st>>>(epi, f, u, pairs);
      e = cudaGetLastError();
      return e == cudaSuccess ? ILS_OK : cuda_fail(e, "output stage launch");
    }
    if ((e = cudaMemcpyAsync(u, u0 ? u0 : f, bytes, cudaMemcpyDeviceToDevice, st))) return cuda_fail(e, "copy");
    e = host_out(pl, k, 0, pl->C, st);
    return e == cudaSuccess ? ILS_OK : cuda_fail(e, "D2H copy");
  }
  ils_status s;
  if (!pl->profiling && pl->nsplit > 1) {
    if ((e = cudaEventRecord(pl->fork_join[0], st))) return cuda_fail(e, "event");
    for (int g = 0; g < pl->nsplit; ++g) {
      const int c0 = g * pl->C / pl->nsplit, c1 = (g + 1) * pl->C / pl->nsplit;
      cudaStream_t sg = pl->side[g];
      if ((e = cudaStreamWaitEvent(sg, pl->fork_join[0], 0))) return cuda_fail(e, "stream wait");
      if (k.f_host != nullptr) {
        // one input copy at a time, group by group, so that group 0 starts computing first
        cudaEvent_t* h2d = &pl->fork_join[1 + pl->nsplit];
        if ((g > 0 && (e = cudaStreamWaitEvent(sg, h2d[g - 1], 0))) || (e = host_in(pl, k, c0, c1 - c0, sg)) ||
            (e = cudaEventRecord(h2d[g], sg)))
          return cuda_fail(e, "H2D copy");
      }
      if ((s = enqueue_ils(pl, c0, c1 - c0, f, u0, u, ckpt, sg, epi, nullptr))) return s;
      if ((e = host_out(pl, k, c0, c1 - c0, sg))) return cuda_fail(e, "D2H copy");
      if ((e = cudaEventRecord(pl->fork_join[1 + g], sg)) || (e = cudaStreamWaitEvent(st, pl->fork_join[1 + g], 0)))
        return cuda_fail(e, "join");
    }
    return ILS_OK;
  }
  int slot = 0;
  if ((e = host_in(pl, k, 0, pl->C, st))) return cuda_fail(e, "H2D copy");
  if ((s = enqueue_ils(pl, 0, pl->C, f, u0, u, ckpt, st, epi, pl->profiling ? &slot : nullptr))) return s;
  if ((e = mark(pl, slot, -1, st))) return cuda_fail(e, "event");
  if ((e = host_out(pl, k, 0, pl->C, st))) return cuda_fail(e, "D2H copy");
  if (pl->profiling) {
    // accumulate this call's launch durations (waits for the call to finish)
    if ((e = cudaEventSynchronize(pl->ev[slot]))) return cuda_fail(e, "cudaEventSynchronize");
    for (int i = 0; i < slot; ++i) {
      float ms = 0.0f;
      if ((e = cudaEventElapsedTime(&ms, pl->ev[i], pl->ev[i + 1]))) return cuda_fail(e, "cudaEventElapsedTime");
      pl->prof_ms[pl->ev_kind[i]] += ms;
      pl->prof_launches[pl->ev_kind[i]] += 1;
    }
  }
  return ILS_OK;
}

}  // namespace

namespace ils {
// exp(-2 pi i t / L) for t = 0..L-1 (double precision, rounded once).
std::vector<float2> unit_roots(int L) {
  std::vector<float2> v(L);
  for (int t = 0; t < L; ++t) {
    const double a = -2.0 * M_PI * (double)t / (double)L;
    v[t] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  return v;
}

std::vector<float2> row_twiddles(int W) {
  const int M = W / 2;
  std::vector<float2> v = unit_roots(W);
  v.resize(row_twiddle_count(W), make_float2(0.0f, 0.0f));
  const int S = four_step_lanes(M);
  for (int t = 0; t < M; ++t) {
    const int k2 = t / S, n1 = t % S;
    v[(size_t)W + t] = v[(size_t)(2 * n1 * k2) % W];  // exp(-2 pi i n1 k2 / M)
  }
  return v;
}

bool pdl_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("ILS_PDL");
    return e != nullptr && e[0] == '1';
  }();
  return on;
}

void record_cuda_error(const char* where, cudaError_t e) {
  g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
}

// Algorithm 1 from u0 (f when null) through the plan with an output stage and optional
// caller-owned checkpoints (the warm-started smoother's call; no argument checks here).
int run_plan_epilogue(ils_plan* pl, const float* f, const float* u0, float* u, float* ckpt, const Epilogue& epi,
                      cudaStream_t st) {
  return (int)run_ils(pl, f, u0, u, ckpt, st, epi);
}
}  // namespace ils

extern "C" {

const char* ils_status_string(ils_status s) {
  switch (s) {
    case ILS_OK: return "ILS_OK";
    case ILS_ERR_INVALID_ARG: return "ILS_ERR_INVALID_ARG";
    case ILS_ERR_UNSUPPORTED_SIZE: return "ILS_ERR_UNSUPPORTED_SIZE";
    case ILS_ERR_OOM: return "ILS_ERR_OOM";
    case ILS_ERR_CUDA: return "ILS_ERR_CUDA";
    case ILS_ERR_TIMEOUT: return "ILS_ERR_TIMEOUT";
    case ILS_ERR_FALLBACK_TAKEN: return "ILS_ERR_FALLBACK_TAKEN";
  }
  return "ILS_ERR_UNKNOWN";
}

const char* ils_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

namespace {

// Shared by both penalties: validates the shape, allocates and fills the tables.
// mp holds the penalty's Eq. 7 / Eq. 19 parameters; c (double) builds the Eq. 9 tables and
// its FP32 rounding goes to the kernels; half_lambda is set here.
ils_status create_plan(int H, int W, int C, float lambda, int N, MuParams mp, double c, float p, float eps,
                       ils_plan** out) {
  if (H < 2 || W < 2 || H > 8192 || W > 8192 || (W & 1) || !smooth_235(H) || !smooth_235(W))
    return ILS_ERR_UNSUPPORTED_SIZE;
  mp.c = (float)c;
  if (!std::isfinite(c) || (size_t)C * H * W > (size_t)1 << 31) return ILS_ERR_UNSUPPORTED_SIZE;

  ils_plan* pl = new (std::nothrow) ils_plan();
  if (pl == nullptr) return ILS_ERR_OOM;
  g_alloc_count = 0;
  pl->H = H; pl->W = W; pl->C = C; pl->N = N;
  pl->lambda = lambda; pl->p = p; pl->eps = eps; pl->c = (float)c;
  pl->desc.H = H; pl->desc.W = W; pl->desc.C = C;
  const int M = W / 2;
  if (!make_fft_plan(M, &pl->desc.planM) || !make_fft_plan(H, &pl->desc.planH) || !pick_geometry(H, W, &pl->geo)) {
    delete pl;
    return ILS_ERR_UNSUPPORTED_SIZE;
  }
  pl->mp = mp;
  pl->mp.half_lambda = 0.5f * lambda;

  cudaError_t e;
  if ((e = cudaGetDevice(&pl->device))) { delete pl; return cuda_fail(e, "cudaGetDevice"); }
  if ((e = set_kernel_attributes())) { delete pl; return cuda_fail(e, "cudaFuncSetAttribute"); }

  const size_t plane = (size_t)C * H * M;
  ils_status s;
  if ((s = dev_alloc((void**)&pl->spec[0], plane * sizeof(float2))) ||
      (s = dev_alloc((void**)&pl->spec[1], plane * sizeof(float2))) ||
      (s = dev_alloc((void**)&pl->tab.twW, row_twiddle_count(W) * sizeof(float2))) ||
      (s = dev_alloc((void**)&pl->tab.twH, col_twiddle_count(H) * sizeof(float2))) ||
      (s = dev_alloc((void**)&pl->tab.ax, (size_t)(M + 1) * sizeof(float))) ||
      (s = dev_alloc((void**)&pl->tab.by, (size_t)H * sizeof(float)))) {
    free_plan_memory(pl);
    delete pl;
    return s;
  }
  // Eq. 9 denominator, separable: 1 + (lambda c / 2)(|F grad_x|^2 + |F grad_y|^2) with
  // |F grad|^2 = 4 sin^2(pi k / n); stored as ax[k] + by[l], each lambda c * 2 sin^2.
  std::vector<float> ax(M + 1), by(H);
  for (int k = 0; k <= M; ++k) {
    const double s1 = std::sin(M_PI * (double)k / (double)W);
    ax[k] = (float)(2.0 * (double)lambda * c * s1 * s1);
  }
  for (int l = 0; l < H; ++l) {
    const double s1 = std::sin(M_PI * (double)l / (double)H);
    by[l] = (float)(2.0 * (double)lambda * c * s1 * s1);
  }
  std::vector<float2> tw = row_twiddles(W), th = unit_roots(H);
  if ((e = cudaMemcpy(pl->tab.twW, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(pl->tab.twH, th.data(), th.size() * sizeof(float2), cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(pl->tab.ax, ax.data(), ax.size() * sizeof(float), cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(pl->tab.by, by.data(), by.size() * sizeof(float), cudaMemcpyHostToDevice)) ||
      (e = build_col_twiddles(H, pl->tab.twH, 0)) || (e = build_row_twiddles(W, pl->tab.twW, 0)) ||
      (e = cudaStreamSynchronize(0))) {
    free_plan_memory(pl);
    delete pl;
    return cuda_fail(e, "tables");
  }
  // 2..8 channels: one internal stream per channel (at most 4); ILS_SPLIT=0 keeps one stream
  const char* split = std::getenv("ILS_SPLIT");
  pl->nsplit = (C >= 2 && C <= 8 && !(split != nullptr && split[0] == '0')) ? std::min(C, 4) : 1;
  for (int k = 0; k < pl->nsplit; ++k) {
    cudaStream_t x;
    if ((e = cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking))) {
      free_plan_memory(pl);
      delete pl;
      return cuda_fail(e, "cudaStreamCreate");
    }
    pl->side.push_back(x);
  }
  for (int k = 0; k < (pl->nsplit > 1 ? 2 * pl->nsplit + 1 : 0); ++k) {
    cudaEvent_t x;
    if ((e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming))) {
      free_plan_memory(pl);
      delete pl;
      return cuda_fail(e, "cudaEventCreate");
    }
    pl->fork_join.push_back(x);
  }
  *out = pl;
  return ILS_OK;
}

}  // namespace

extern "C" {

ils_status ils_plan_create(int H, int W, int C, float lambda, float p, float eps, int N, ils_plan** out) {
  if (out == nullptr) return ILS_ERR_INVALID_ARG;
  *out = nullptr;
  if (C < 1 || N < 0 || !(lambda >= 0.0f) || !std::isfinite(lambda) || !(eps > 0.0f) || !std::isfinite(eps) ||
      !((p > 0.0f && p <= 1.0f) || p == 2.0f))
    return ILS_ERR_INVALID_ARG;
  MuParams mp;
  mp.p = p;
  mp.eps = eps;
  mp.a = p / 2.0f - 1.0f;
  const double c = (double)p * std::pow((double)eps, (double)p / 2.0 - 1.0);  // c = c0 (Eq. 11)
  return create_plan(H, W, C, lambda, N, mp, c, p, eps, out);
}

ils_status ils_plan_create_hqs(int H, int W, int C, float lambda, float beta0, float kappa, int N, ils_plan** out) {
  if (out == nullptr) return ILS_ERR_INVALID_ARG;
  *out = nullptr;
  if (beta0 <= 0.0f) beta0 = 2.0f * lambda;  // the paper's beta_0 = 2 lambda
  if (C < 1 || N < 0 || !(lambda > 0.0f) || !std::isfinite(lambda) || !(beta0 > 0.0f) || !std::isfinite(beta0) ||
      !(kappa >= 1.0f) || !std::isfinite(kappa) || !std::isfinite((double)beta0 * std::pow((double)kappa, N)))
    return ILS_ERR_INVALID_ARG;
  MuParams mp;
  mp.pen = 2;
  mp.p = 0.0f;
  mp.eps = 1.0f;
  ils_status s = create_plan(H, W, C, lambda, N, mp, 0.0, 0.0f, 1.0f, out);
  if (s != ILS_OK) return s;
  ils_plan* pl = *out;
  const int M = W / 2;
  const size_t per = (size_t)M + 1 + H;
  std::vector<float> tabs(per * (size_t)(N > 0 ? N : 1));
  double beta = beta0;
  for (int n = 0; n < N; ++n, beta *= kappa) {
    MuParams m = pl->mp;
    m.half_lambda = (float)beta;              // Q2 of Eq. 14: u = A_n^{-1}(f + beta_n D^T mu)
    m.thr = (float)(lambda / (2.0 * beta));   // Q1: soft threshold at lambda / (2 beta_n)
    pl->mp_iter.push_back(m);
    for (int k = 0; k <= M; ++k) {
      const double s1 = std::sin(M_PI * (double)k / (double)W);
      tabs[n * per + k] = (float)(4.0 * beta * s1 * s1);  // beta_n |F grad_x|^2
    }
    for (int l = 0; l < H; ++l) {
      const double s1 = std::sin(M_PI * (double)l / (double)H);
      tabs[n * per + M + 1 + l] = (float)(4.0 * beta * s1 * s1);
    }
  }
  cudaError_t e;
  if ((s = dev_alloc((void**)&pl->iter_tab, tabs.size() * sizeof(float))) ||
      (e = cudaMemcpy(pl->iter_tab, tabs.data(), tabs.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess) {
    ils_plan_destroy(pl);
    *out = nullptr;
    return s != ILS_OK ? s : cuda_fail(e, "cudaMemcpy tables");
  }
  return ILS_OK;
}

ils_status ils_plan_create_welsch(int H, int W, int C, float lambda, float gamma, int N, ils_plan** out) {
  if (out == nullptr) return ILS_ERR_INVALID_ARG;
  *out = nullptr;
  if (C < 1 || N < 0 || !(lambda >= 0.0f) || !std::isfinite(lambda) || !(gamma > 0.0f) || !std::isfinite(gamma))
    return ILS_ERR_INVALID_ARG;
  const double inv2g2 = 1.0 / (2.0 * (double)gamma * (double)gamma);
  if (!std::isfinite(inv2g2) || inv2g2 > 1e30) return ILS_ERR_INVALID_ARG;
  MuParams mp;
  mp.p = 0.0f;
  mp.eps = 1.0f;
  mp.a = 0.0f;
  mp.pen = 1;
  mp.wbeta = (float)(inv2g2 / std::log(2.0));  // exp(-x^2/(2 gamma^2)) = 2^(-wbeta x^2)
  mp.winv2g2 = (float)inv2g2;
  return create_plan(H, W, C, lambda, N, mp, 2.0, 0.0f, 1.0f, out);  // c = c0 = 2 (Eq. 20)
}

ils_status ils_plan_destroy(ils_plan* pl) {
  if (pl == nullptr) return ILS_OK;
  cudaError_t e = cudaDeviceSynchronize();
  free_plan_memory(pl);
  delete pl;
  return e == cudaSuccess ? ILS_OK : cuda_fail(e, "cudaDeviceSynchronize");
}

float ils_plan_c(const ils_plan* pl) { return pl ? pl->c : -1.0f; }

ils_status ils_set_profiling(ils_plan* pl, int on) {
  if (pl == nullptr) return ILS_ERR_INVALID_ARG;
  for (int k = 0; k < ILS_KERNEL_KINDS; ++k) {
    pl->prof_ms[k] = 0.0;
    pl->prof_launches[k] = 0;
  }
  if (!on) {
    destroy_events(pl);
    pl->profiling = false;
    return ILS_OK;
  }
  if (pl->ev.empty()) {
    const int slots = 2 * pl->N + 2;
    pl->ev.assign(slots, nullptr);
    pl->ev_kind.assign(slots, -1);
    for (int i = 0; i < slots; ++i) {
      cudaError_t e = cudaEventCreate(&pl->ev[i]);
      if (e != cudaSuccess) {
        destroy_events(pl);
        return cuda_fail(e, "cudaEventCreate");
      }
    }
  }
  pl->profiling = true;
  return ILS_OK;
}

ils_status ils_get_profile(const ils_plan* pl, double* ms, long long* launches) {
  if (pl == nullptr || ms == nullptr || launches == nullptr) return ILS_ERR_INVALID_ARG;
  for (int k = 0; k < ILS_KERNEL_KINDS; ++k) {
    ms[k] = pl->prof_ms[k];
    launches[k] = pl->prof_launches[k];
  }
  return ILS_OK;
}

ils_status ils_smooth_from(ils_plan* pl, const float* f, const float* u0, float* u, void* stream) {
  if (pl == nullptr || f == nullptr || u == nullptr) return ILS_ERR_INVALID_ARG;
  const size_t bytes = (size_t)pl->C * pl->H * pl->W * sizeof(float);
  if (overlaps(f, u, bytes) || (u0 != nullptr && overlaps(u0, u, bytes))) return ILS_ERR_INVALID_ARG;
  float* ck = nullptr;
  if (pl->ckpt_own != nullptr) {
    ck = pl->ckpt_own;
    pl->ckpt_valid = false;  // until the call is enqueued
  }
  const ils_status s = run_ils(pl, f, u0, u, ck, static_cast<cudaStream_t>(stream));
  if (ck != nullptr && s == ILS_OK) {
    pl->ckpt_f = f;
    pl->ckpt_u0 = u0 == f ? nullptr : u0;
    pl->ckpt_valid = true;
  }
  return s;
}

ils_status ils_set_checkpointing(ils_plan* pl, int on) {
  if (pl == nullptr || !pl->mp_iter.empty()) return ILS_ERR_INVALID_ARG;  // no adjoint of the splitting
  pl->ckpt_valid = false;
  if (!on) {
    if (pl->ckpt_own != nullptr) {
      const cudaError_t e = cudaDeviceSynchronize();  // the buffer may still be written
      cudaFree(pl->ckpt_own);
      pl->ckpt_own = nullptr;
      if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
    }
    return ILS_OK;
  }
  if (pl->ckpt_own != nullptr || pl->N == 0) return ILS_OK;
  return dev_alloc((void**)&pl->ckpt_own, (size_t)pl->N * pl->C * pl->H * pl->W * sizeof(float));
}

ils_status ils_smooth_checkpointed(ils_plan* pl, const float* f, const float* u0, float* u, float* ckpt,
                                   void* stream) {
  if (pl == nullptr || f == nullptr || u == nullptr || (ckpt == nullptr && pl->N > 0)) return ILS_ERR_INVALID_ARG;
  const size_t bytes = (size_t)pl->C * pl->H * pl->W * sizeof(float);
  const size_t cbytes = bytes * (size_t)pl->N;
  if (overlaps(f, u, bytes) || (u0 != nullptr && overlaps(u0, u, bytes))) return ILS_ERR_INVALID_ARG;
  if (pl->N > 0 && (overlaps2(ckpt, cbytes, f, bytes) || overlaps2(ckpt, cbytes, u, bytes) ||
                    (u0 != nullptr && overlaps2(ckpt, cbytes, u0, bytes))))
    return ILS_ERR_INVALID_ARG;
  return run_ils(pl, f, u0, u, pl->N > 0 ? ckpt : nullptr, static_cast<cudaStream_t>(stream));
}

ils_status ils_backward_ckpt(ils_plan* pl, const float* ckpt, const float* grad_u, float* grad_f, float* grad_u0,
                             void* stream) {
  if (pl == nullptr || grad_u == nullptr || grad_f == nullptr || (ckpt == nullptr && pl->N > 0) ||
      !pl->mp_iter.empty())  // no adjoint for half-quadratic splitting
    return ILS_ERR_INVALID_ARG;
  const size_t n = (size_t)pl->C * pl->H * pl->W;
  const size_t bytes = n * sizeof(float);
  if (overlaps(grad_u, grad_f, bytes) || (grad_u0 != nullptr && (overlaps(grad_u0, grad_f, bytes) ||
                                                               overlaps(grad_u0, grad_u, bytes))))
    return ILS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (pl->N == 0) {
    // u = u^0: the whole gradient belongs to u^0 (= f unless a separate u^0 gradient is asked for)
    if (grad_u0 != nullptr) {
      if ((e = cudaMemcpyAsync(grad_u0, grad_u, bytes, cudaMemcpyDeviceToDevice, st))) return cuda_fail(e, "copy");
      if ((e = cudaMemsetAsync(grad_f, 0, bytes, st))) return cuda_fail(e, "memset");
    } else if ((e = cudaMemcpyAsync(grad_f, grad_u, bytes, cudaMemcpyDeviceToDevice, st))) {
      return cuda_fail(e, "copy");
    }
    return ILS_OK;
  }
  // spectrum of grad_u (a row pass with lambda = 0 is a plain forward row FFT), then r = A^-1 grad_u
  MuParams plain = pl->mp;
  plain.half_lambda = 0.0f;
  ImageDesc d = pl->desc;  // first launch in caller order, the rest chained (programmatic)
  if ((e = launch_row_forward(d, pl->geo, pl->tab, plain, grad_u, grad_u, nullptr, pl->spec[0], nullptr, st)))
    return cuda_fail(e, "row pass launch");
  d.pdl = pdl_enabled();
  if ((e = launch_col_solve(d, pl->geo, pl->tab, pl->spec[0], st))) return cuda_fail(e, "column pass launch");
  int cur = 0;
  for (int it = pl->N - 1; it >= 0; --it) {
    const bool last = it == 0;
    if ((e = launch_row_adjoint(d, pl->geo, pl->tab, pl->mp, pl->spec[cur], ckpt + (size_t)it * n, grad_f,
                                it == pl->N - 1, grad_u0, last, pl->spec[cur ^ 1], st)))
      return cuda_fail(e, "adjoint row pass launch");
    if (!last) {
      if ((e = launch_col_solve(d, pl->geo, pl->tab, pl->spec[cur ^ 1], st)))
        return cuda_fail(e, "column pass launch");
      cur ^= 1;
    }
  }
  return ILS_OK;
}

ils_status ils_backward(ils_plan* pl, const float* f, const float* grad_u, float* grad_f, void* stream) {
  if (pl == nullptr || f == nullptr || grad_u == nullptr || grad_f == nullptr) return ILS_ERR_INVALID_ARG;
  // the checkpoints must be those of a forward call on this f
  if (pl->N > 0 && (pl->ckpt_own == nullptr || !pl->ckpt_valid || pl->ckpt_f != f)) return ILS_ERR_INVALID_ARG;
  const size_t bytes = (size_t)pl->C * pl->H * pl->W * sizeof(float);
  if (overlaps(grad_f, f, bytes)) return ILS_ERR_INVALID_ARG;
  // u^0 = f: dL/du^0 joins dL/df; a separate warm start u^0 keeps only the direct part
  float* gu0 = nullptr;
  if (pl->N > 0 && pl->ckpt_u0 != nullptr) {
    if (pl->stage_u == nullptr) {
      const ils_status s = dev_alloc((void**)&pl->stage_u, bytes);
      if (s != ILS_OK) return s;
    }
    gu0 = pl->stage_u;
  }
  return ils_backward_ckpt(pl, pl->ckpt_own, grad_u, grad_f, gu0, stream);
}

ils_status ils_smooth(ils_plan* pl, const float* f, float* u, void* stream) {
  if (pl == nullptr || f == nullptr || u == nullptr) return ILS_ERR_INVALID_ARG;
  return ils_smooth_from(pl, f, nullptr, u, stream);
}

ils_status ils_smooth_enhance(ils_plan* pl, const float* f, float* out, float k, void* stream) {
  if (pl == nullptr || f == nullptr || out == nullptr || !std::isfinite(k)) return ILS_ERR_INVALID_ARG;
  const size_t bytes = (size_t)pl->C * pl->H * pl->W * sizeof(float);
  if (overlaps(f, out, bytes)) return ILS_ERR_INVALID_ARG;
  Epilogue epi;
  epi.mode = 1;
  epi.s = 1.0f - k;
  epi.f = f;
  return run_ils(pl, f, nullptr, out, nullptr, static_cast<cudaStream_t>(stream), epi);
}

ils_status ils_smooth_luma(ils_plan* pl, const float* rgb, float* out, float k, void* stream) {
  if (pl == nullptr || rgb == nullptr || out == nullptr || pl->C != 1 || !std::isfinite(k))
    return ILS_ERR_INVALID_ARG;
  const size_t n = (size_t)pl->H * pl->W;
  if (overlaps(rgb, out, 3 * n * sizeof(float))) return ILS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (pl->N == 0) {  // u = Y: out = rgb
    e = cudaMemcpyAsync(out, rgb, 3 * n * sizeof(float), cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? ILS_OK : cuda_fail(e, "cudaMemcpyAsync");
  }
  if (pl->luma == nullptr) {
    ils_status s = dev_alloc((void**)&pl->luma, n * sizeof(float));
    if (s != ILS_OK) return s;
  }
  luma_kernel<<<(int)std::min<size_t>((n + 255) / 256, 4096), 256, 0, st>>>(rgb, pl->luma, n);
  if ((e = cudaGetLastError())) return cuda_fail(e, "luma kernel launch");
  Epilogue epi;
  epi.mode = 2;
  epi.s = 1.0f - k;
  epi.f = pl->luma;
  epi.rgb = rgb;
  epi.plane2 = n / 2;
  return run_ils(pl, pl->luma, nullptr, out, nullptr, st, epi);
}

ils_status ils_smooth_hwc(ils_plan* pl, const float* f_hwc, float* u_hwc, void* stream) {
  if (pl == nullptr || f_hwc == nullptr || u_hwc == nullptr) return ILS_ERR_INVALID_ARG;
  const size_t hw = (size_t)pl->H * pl->W, n = (size_t)pl->C * hw;
  if (n / 2 >= ((size_t)1 << 32)) return ILS_ERR_UNSUPPORTED_SIZE;  // 32-bit pair index of the output stage
  if (overlaps(f_hwc, u_hwc, n * sizeof(float))) return ILS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (pl->N == 0) {
    e = cudaMemcpyAsync(u_hwc, f_hwc, n * sizeof(float), cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? ILS_OK : cuda_fail(e, "cudaMemcpyAsync");
  }
  if (pl->stage_f == nullptr) {
    ils_status s = dev_alloc((void**)&pl->stage_f, n * sizeof(float));
    if (s != ILS_OK) return s;
  }
  hwc_to_planar_kernel<<<grid_for(hw), 256, 0, st>>>(f_hwc, pl->stage_f, pl->C, hw);
  if ((e = cudaGetLastError())) return cuda_fail(e, "interleaved load launch");
  Epilogue epi;
  epi.mode = 3;
  epi.dst = u_hwc;
  epi.C = pl->C;
  epi.plane2 = hw / 2;
  // the planar image is the only planar buffer; the output stage writes u_hwc instead of it
  return run_ils(pl, pl->stage_f, nullptr, pl->stage_f, nullptr, st, epi);
}

ils_status ils_log_luma(const float* rgb, float* l, int H, int W, void* stream) {
  if (rgb == nullptr || l == nullptr || H < 1 || W < 1) return ILS_ERR_INVALID_ARG;
  const size_t n = (size_t)H * W;
  if (overlaps2(rgb, 3 * n * sizeof(float), l, n * sizeof(float))) return ILS_ERR_INVALID_ARG;
  log_luma_kernel<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(rgb, l, n);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ILS_OK : cuda_fail(e, "log-luminance launch");
}

ils_status ils_tonemap_log(ils_plan* pl, const float* rgb, float* out, float s, float k, float o, void* stream) {
  if (pl == nullptr || rgb == nullptr || out == nullptr || pl->C != 1 || !std::isfinite(s) || !std::isfinite(k) ||
      !std::isfinite(o))
    return ILS_ERR_INVALID_ARG;
  const size_t n = (size_t)pl->H * pl->W;
  if (overlaps(rgb, out, 3 * n * sizeof(float))) return ILS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (pl->luma == nullptr) {
    ils_status r = dev_alloc((void**)&pl->luma, n * sizeof(float));
    if (r != ILS_OK) return r;
  }
  log_luma_kernel<<<grid_for(n), 256, 0, st>>>(rgb, pl->luma, n);
  cudaError_t e;
  if ((e = cudaGetLastError())) return cuda_fail(e, "log-luminance launch");
  // l' = s b + k (l - b) and out_c = rgb_c exp(l' - l + o) = rgb_c exp((k - 1) l + (s - k) b + o)
  Epilogue epi;
  epi.mode = 4;
  epi.a = k - 1.0f;
  epi.s = s - k;
  epi.o = o;
  epi.f = pl->luma;
  epi.rgb = rgb;
  epi.plane2 = n / 2;
  return run_ils(pl, pl->luma, nullptr, out, nullptr, st, epi);
}

ils_status ils_gaussian_blur(const float* f, float* out, int H, int W, int C, float sigma, void* stream) {
  if (f == nullptr || out == nullptr || H < 1 || W < 1 || C < 1 || C > 65535 || !(sigma >= 0.0f) || sigma > 5.0f)
    return ILS_ERR_INVALID_ARG;
  if (overlaps(f, out, (size_t)C * H * W * sizeof(float))) return ILS_ERR_INVALID_ARG;
  const cudaError_t e = launch_gaussian_blur(f, out, H, W, C, sigma, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? ILS_OK : cuda_fail(e, "Gaussian blur launch");
}

ils_status ils_smooth_presmoothed(ils_plan* pl, const float* f, float* u, float sigma, void* stream) {
  if (pl == nullptr || f == nullptr || u == nullptr || !(sigma >= 0.0f) || sigma > 5.0f) return ILS_ERR_INVALID_ARG;
  const size_t bytes = (size_t)pl->C * pl->H * pl->W * sizeof(float);
  if (overlaps(f, u, bytes)) return ILS_ERR_INVALID_ARG;
  if (pl->stage_f == nullptr) {
    const ils_status s = dev_alloc((void**)&pl->stage_f, bytes);
    if (s != ILS_OK) return s;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const cudaError_t e = launch_gaussian_blur(f, pl->stage_f, pl->H, pl->W, pl->C, sigma, st);
  if (e != cudaSuccess) return cuda_fail(e, "Gaussian blur launch");
  return run_ils(pl, pl->stage_f, nullptr, u, nullptr, st);
}

ils_status ils_smooth_host(ils_plan* pl, const float* f_host, float* u_host, void* stream) {
  if (pl == nullptr || f_host == nullptr || u_host == nullptr) return ILS_ERR_INVALID_ARG;
  const size_t bytes = (size_t)pl->C * pl->H * pl->W * sizeof(float);
  ils_status s;
  if (pl->stage_f == nullptr) {
    if ((s = dev_alloc((void**)&pl->stage_f, bytes))) return s;
  }
  if (pl->stage_u == nullptr) {
    if ((s = dev_alloc((void**)&pl->stage_u, bytes))) return s;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  // the copies run inside the launch sequence, per channel group (launch_all)
  if ((s = run_ils(pl, pl->stage_f, nullptr, pl->stage_u, nullptr, st, Epilogue(), f_host, u_host))) return s;
  if ((e = cudaStreamSynchronize(st))) return cuda_fail(e, "cudaStreamSynchronize");
  return ILS_OK;
}

}  // extern "C"
