// Batched smoothing of frames of uneven size in one CUDA-graph launch.
//
// Frames are grouped into size classes (H, W, C); a class shares the FFT plans, launch
// geometry and twiddle tables, while each frame keeps its own lambda, p, eps, N (its
// Eq. 7 parameters and its Eq. 9 denominator tables).  Frames are spread over parallel
// graph branches by longest-processing-time-first on pixel count; a branch runs its frames
// one after another in one pair of spectrum workspaces.  The whole batch - every pass of
// every frame - is captured once into a CUDA graph, so a run is a single graph launch.
// An optional autotuner picks, per class, among the compile-time tile shapes and the
// generic kernels by timing them, and can keep its choices in a file.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ils.h"
#include "ils_internal.h"

using namespace ils;

namespace ils {
std::vector<float2> unit_roots(int L);  // exp(-2 pi i t / L), t < L (ils_capi.cu)
}

namespace {

struct BatchClass {
  int H, W, C;
  ImageDesc desc;
  Geometry geo;
  float2* twW = nullptr;
  float2* twH = nullptr;
  size_t elems() const { return (size_t)C * H * W; }
};

struct BatchFrame {
  int cls, N;
  MuParams mp;
  float* ax = nullptr;
  float* by = nullptr;
  const float* f;
  float* u;
  int branch;
};

bool smooth_235(int n) {
  if (n < 1) return false;
  for (int r : {2, 3, 5})
    while (n % r == 0) n /= r;
  return n == 1;
}

template <typename T>
cudaError_t upload(T** dst, const std::vector<T>& v) {
  cudaError_t e = cudaMalloc((void**)dst, v.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

// All passes of Algorithm 1 for one frame on `st`.
cudaError_t enqueue_frame(const BatchClass& c, const BatchFrame& fr, float2* s0, float2* s1, cudaStream_t st) {
  Tables t{c.twW, c.twH, fr.ax, fr.by};
  cudaError_t e;
  if (fr.N == 0) return cudaMemcpyAsync(fr.u, fr.f, c.elems() * sizeof(float), cudaMemcpyDeviceToDevice, st);
  float2* sp[2] = {s0, s1};
  ImageDesc d = c.desc;  // the frame's first launch in stream order, the rest chained (programmatic)
  for (int it = 0; it < fr.N; ++it) {
    float2* out = sp[it & 1];
    const float2* in = it == 0 ? nullptr : sp[(it - 1) & 1];
    d.pdl = it > 0 && pdl_enabled();
    if ((e = launch_row_forward(d, c.geo, t, fr.mp, fr.f, nullptr, in, out, nullptr, st))) return e;
    d.pdl = pdl_enabled();
    if ((e = launch_col_solve(d, c.geo, t, out, st))) return e;
  }
  return launch_row_inverse(d, c.geo, t, sp[(fr.N - 1) & 1], fr.u, st);
}

ils_status fail(cudaError_t e, const char* where) {
  record_cuda_error(where, e);
  return ILS_ERR_CUDA;
}

// ---------------------------------------------------------------- autotuner

std::string device_name() {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
  std::string n = prop.name;
  for (char& ch : n)
    if (ch == ' ') ch = '_';
  return n;
}

// Cache file lines: "<device> <H> <W> <C> <row variant> <col variant>": row variant 1000 + w
// for warp-per-row entry w, else a block-per-strip entry (-1 = generic kernels).
bool cache_lookup(const char* path, const std::string& dev, int H, int W, int C, int* rv, int* cv) {
  if (path == nullptr) return false;
  FILE* fp = std::fopen(path, "r");
  if (fp == nullptr) return false;
  char name[256];
  int h, w, c, r, k;
  bool found = false;
  while (std::fscanf(fp, "%255s %d %d %d %d %d", name, &h, &w, &c, &r, &k) == 6) {
    if (dev == name && h == H && w == W && c == C) {
      *rv = r;
      *cv = k;
      found = true;
    }
  }
  std::fclose(fp);
  return found;
}

void cache_store(const char* path, const std::string& dev, int H, int W, int C, int rv, int cv) {
  if (path == nullptr) return;
  FILE* fp = std::fopen(path, "a");
  if (fp == nullptr) return;
  std::fprintf(fp, "%s %d %d %d %d %d\n", dev.c_str(), H, W, C, rv, cv);
  std::fclose(fp);
}

// Median time (ms) over kTuneRuns separately timed N=1 smoothings of a class-sized frame with
// geometry g (after two untimed runs): one slow sample - another tenant's burst, a clock step -
// does not decide the choice.
constexpr int kTuneRuns = 7;
float time_geometry(const BatchClass& c, const Geometry& g, const BatchFrame& proto, float* f, float* u, float2* s0,
                    float2* s1, cudaStream_t st) {
  BatchClass cc = c;
  cc.geo = g;
  BatchFrame fr = proto;
  fr.N = 1;
  fr.f = f;
  fr.u = u;
  cudaEvent_t ev[kTuneRuns + 1];
  int made = 0;
  for (; made <= kTuneRuns; ++made)
    if (cudaEventCreate(&ev[made]) != cudaSuccess) break;
  float ms = 1e30f;
  if (made == kTuneRuns + 1) {
    for (int i = 0; i < 2; ++i) enqueue_frame(cc, fr, s0, s1, st);
    cudaEventRecord(ev[0], st);
    for (int i = 0; i < kTuneRuns; ++i) {
      enqueue_frame(cc, fr, s0, s1, st);
      cudaEventRecord(ev[i + 1], st);
    }
    if (cudaEventSynchronize(ev[kTuneRuns]) == cudaSuccess) {
      std::vector<float> t(kTuneRuns, 1e30f);
      for (int i = 0; i < kTuneRuns; ++i) cudaEventElapsedTime(&t[i], ev[i], ev[i + 1]);
      std::nth_element(t.begin(), t.begin() + kTuneRuns / 2, t.end());
      ms = t[kTuneRuns / 2];
    }
  }
  for (int i = 0; i < made; ++i) cudaEventDestroy(ev[i]);
  if (cudaGetLastError() != cudaSuccess) return 1e30f;
  return ms;
}

// Pick the row and column kernels for a class: every compile-time tile shape for its
// lengths and the generic kernels, timed one knob at a time.
ils_status autotune_class(BatchClass& c, const BatchFrame& proto) {
  const char* path = std::getenv("ILS_AUTOTUNE_CACHE");
  const std::string dev = device_name();
  int rv = -2, cv = -2;
  int rows[8], cols[8];
  int nr = fixed_row_variants(c.W / 2, rows, 7), nc = fixed_col_variants(c.H, cols, 7);
  rows[nr++] = -1;
  cols[nc++] = -1;
  int wl[8];
  const int nwl = warp_row_variants(c.W / 2, wl, 8);
  if (cache_lookup(path, dev, c.H, c.W, c.C, &rv, &cv) && std::find(cols, cols + nc, cv) != cols + nc) {
    // entries from another build (unknown variant indices) are ignored
    if (rv >= 1000 && std::find(wl, wl + nwl, rv - 1000) != wl + nwl) {
      c.geo.warp_row = rv - 1000;
      c.geo.fixed_col = cv;
      return ILS_OK;
    }
    if (rv < 1000 && std::find(rows, rows + nr, rv) != rows + nr) {
      c.geo.warp_row = -1;
      c.geo.fixed_row = rv;
      c.geo.fixed_col = cv;
      return ILS_OK;
    }
  }
  const size_t n = c.elems();
  float *f = nullptr, *u = nullptr;
  float2 *s0 = nullptr, *s1 = nullptr;
  cudaStream_t st = nullptr;
  cudaError_t e;
  if ((e = cudaMalloc((void**)&f, n * 4)) || (e = cudaMalloc((void**)&u, n * 4)) ||
      (e = cudaMalloc((void**)&s0, n * 4)) || (e = cudaMalloc((void**)&s1, n * 4)) ||
      (e = cudaMemset(f, 0, n * 4)) || (e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking))) {
    cudaFree(f); cudaFree(u); cudaFree(s0); cudaFree(s1);
    return fail(e, "autotune allocation");
  }
  // row candidates: every warp-per-row entry, then (warp kernels off) every block-per-strip
  // entry and the generic kernels; encoded as w (>= 0) for warp entry w, -2 - i for row entry i
  int wv[8];
  const int nw = warp_row_variants(c.W / 2, wv, 8);
  Geometry g = c.geo;
  float best = 1e30f;
  int best_w = g.warp_row, best_r = g.fixed_row;
  for (int i = 0; i < nw + nr; ++i) {
    if (i < nw) {
      g.warp_row = wv[i];
    } else {
      g.warp_row = -1;
      g.fixed_row = rows[i - nw];
    }
    const float ms = time_geometry(c, g, proto, f, u, s0, s1, st);
    if (ms < best) {
      best = ms;
      best_w = g.warp_row;
      best_r = g.fixed_row;
    }
  }
  g.warp_row = best_w;
  g.fixed_row = best_r;
  best = 1e30f;
  int best_c = g.fixed_col;
  for (int i = 0; i < nc; ++i) {
    g.fixed_col = cols[i];
    const float ms = time_geometry(c, g, proto, f, u, s0, s1, st);
    if (ms < best) { best = ms; best_c = cols[i]; }
  }
  c.geo.warp_row = best_w;
  c.geo.fixed_row = best_r;
  c.geo.fixed_col = best_c;
  cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
  cudaFree(f); cudaFree(u); cudaFree(s0); cudaFree(s1);
  cache_store(path, dev, c.H, c.W, c.C, best_w >= 0 ? 1000 + best_w : best_r, best_c);
  return ILS_OK;
}

}  // namespace

struct ils_batch {
  std::vector<BatchClass> cls;
  std::vector<BatchFrame> fr;
  int nbranch = 0;
  std::vector<float2*> ws;  // 2 per branch
  std::vector<cudaStream_t> streams;
  cudaStream_t origin = nullptr;
  std::vector<cudaEvent_t> events;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

void release(ils_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (cudaEvent_t e : b->events) cudaEventDestroy(e);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  if (b->origin) cudaStreamDestroy(b->origin);
  for (float2* p : b->ws) cudaFree(p);
  for (BatchFrame& f : b->fr) {
    cudaFree(f.ax);
    cudaFree(f.by);
  }
  for (BatchClass& c : b->cls) {
    cudaFree(c.twW);
    cudaFree(c.twH);
  }
  delete b;
}

ils_status capture(ils_batch* b) {
  cudaError_t e;
  cudaStream_t o = b->origin;
  if ((e = cudaStreamBeginCapture(o, cudaStreamCaptureModeThreadLocal))) return fail(e, "cudaStreamBeginCapture");
  ils_status s = ILS_OK;
  // fork: every branch stream waits for the origin; join: the origin waits for every branch
  cudaEvent_t fork = b->events[0];
  if ((e = cudaEventRecord(fork, o))) s = fail(e, "cudaEventRecord");
  for (int br = 0; br < b->nbranch && s == ILS_OK; ++br) {
    cudaStream_t st = b->streams[br];
    if ((e = cudaStreamWaitEvent(st, fork, 0))) { s = fail(e, "cudaStreamWaitEvent"); break; }
    for (const BatchFrame& fr : b->fr) {
      if (fr.branch != br) continue;
      if ((e = enqueue_frame(b->cls[fr.cls], fr, b->ws[2 * br], b->ws[2 * br + 1], st))) {
        s = fail(e, "kernel launch during capture");
        break;
      }
    }
    if (s != ILS_OK) break;
    if ((e = cudaEventRecord(b->events[1 + br], st))) { s = fail(e, "cudaEventRecord"); break; }
    if ((e = cudaStreamWaitEvent(o, b->events[1 + br], 0))) { s = fail(e, "cudaStreamWaitEvent"); break; }
  }
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(o, &g);
  if (s != ILS_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) return fail(e, "cudaStreamEndCapture");
  b->graph = g;
  if ((e = cudaGraphInstantiate(&b->exec, g, 0))) return fail(e, "cudaGraphInstantiate");
  return ILS_OK;
}

}  // namespace

extern "C" {

ils_status ils_batch_create(const ils_frame* frames, int count, int flags, ils_batch** out) {
  if (out == nullptr) return ILS_ERR_INVALID_ARG;
  *out = nullptr;
  if (frames == nullptr || count < 1 || (flags & ~ILS_BATCH_AUTOTUNE) != 0) return ILS_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i) {
    const ils_frame& f = frames[i];
    if (f.f == nullptr || f.u == nullptr || f.C < 1 || f.N < 0 || !(f.lambda >= 0.0f) || !std::isfinite(f.lambda) ||
        !(f.eps > 0.0f) || !std::isfinite(f.eps) || !((f.p > 0.0f && f.p <= 1.0f) || f.p == 2.0f))
      return ILS_ERR_INVALID_ARG;
    if (f.H < 2 || f.W < 2 || f.H > 8192 || f.W > 8192 || (f.W & 1) || !smooth_235(f.H) || !smooth_235(f.W))
      return ILS_ERR_UNSUPPORTED_SIZE;
    const size_t bytes = (size_t)f.C * f.H * f.W * sizeof(float);
    const uintptr_t a = reinterpret_cast<uintptr_t>(f.f), b = reinterpret_cast<uintptr_t>(f.u);
    if (a < b + bytes && b < a + bytes) return ILS_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j) {  // outputs must not overlap other frames' inputs or outputs
      const ils_frame& g = frames[j];
      const size_t gb = (size_t)g.C * g.H * g.W * sizeof(float);
      const uintptr_t gu = reinterpret_cast<uintptr_t>(g.u), gf = reinterpret_cast<uintptr_t>(g.f);
      if ((b < gu + gb && gu < b + bytes) || (b < gf + gb && gf < b + bytes) || (gu < a + bytes && a < gu + gb))
        return ILS_ERR_INVALID_ARG;
    }
  }
  ils_batch* B = new (std::nothrow) ils_batch();
  if (B == nullptr) return ILS_ERR_OOM;
  cudaError_t e;
  ils_status s = ILS_OK;
  if ((e = set_kernel_attributes())) { release(B); return fail(e, "cudaFuncSetAttribute"); }
  // size classes
  for (int i = 0; i < count && s == ILS_OK; ++i) {
    const ils_frame& f = frames[i];
    int ci = -1;
    for (int k = 0; k < (int)B->cls.size(); ++k)
      if (B->cls[k].H == f.H && B->cls[k].W == f.W && B->cls[k].C == f.C) ci = k;
    if (ci < 0) {
      BatchClass c;
      c.H = f.H; c.W = f.W; c.C = f.C;
      c.desc.H = f.H; c.desc.W = f.W; c.desc.C = f.C;
      if (!make_fft_plan(f.W / 2, &c.desc.planM) || !make_fft_plan(f.H, &c.desc.planH) ||
          !pick_geometry(f.H, f.W, &c.geo)) {
        s = ILS_ERR_UNSUPPORTED_SIZE;
        break;
      }
      B->cls.push_back(c);
      ci = (int)B->cls.size() - 1;
      std::vector<float2> th = unit_roots(f.H);
      th.resize(col_twiddle_count(f.H));  // stage tables, gathered on the device below
      if ((e = upload(&B->cls[ci].twW, row_twiddles(f.W))) || (e = upload(&B->cls[ci].twH, th)) ||
          (e = build_col_twiddles(f.H, B->cls[ci].twH, 0)) || (e = build_row_twiddles(f.W, B->cls[ci].twW, 0)) ||
          (e = cudaStreamSynchronize(0))) {
        s = fail(e, "class tables");
        break;
      }
    }
    BatchFrame fr;
    fr.cls = ci;
    fr.N = f.N;
    const double c = (double)f.p * std::pow((double)f.eps, (double)f.p / 2.0 - 1.0);
    fr.mp.c = (float)c;
    fr.mp.p = f.p;
    fr.mp.eps = f.eps;
    fr.mp.a = f.p / 2.0f - 1.0f;
    fr.mp.half_lambda = 0.5f * f.lambda;
    fr.f = f.f;
    fr.u = f.u;
    fr.branch = 0;
    // Eq. 9 denominator tables for this frame's lambda c (see ils_plan_create)
    std::vector<float> ax(f.W / 2 + 1), by(f.H);
    for (int k = 0; k <= f.W / 2; ++k) {
      const double s1 = std::sin(M_PI * (double)k / (double)f.W);
      ax[k] = (float)(2.0 * (double)f.lambda * c * s1 * s1);
    }
    for (int l = 0; l < f.H; ++l) {
      const double s1 = std::sin(M_PI * (double)l / (double)f.H);
      by[l] = (float)(2.0 * (double)f.lambda * c * s1 * s1);
    }
    B->fr.push_back(fr);
    if ((e = upload(&B->fr.back().ax, ax)) || (e = upload(&B->fr.back().by, by))) {
      s = fail(e, "frame tables");
      break;
    }
  }
  if (s == ILS_OK && (flags & ILS_BATCH_AUTOTUNE)) {
    for (int k = 0; k < (int)B->cls.size() && s == ILS_OK; ++k) {
      int proto = 0;
      for (int i = 0; i < count; ++i)
        if (B->fr[i].cls == k) proto = i;
      s = autotune_class(B->cls[k], B->fr[proto]);
    }
  }
  if (s != ILS_OK) { release(B); return s; }
  // branches: longest processing time first on pixel count
  const char* nb_env = std::getenv("ILS_BATCH_BRANCHES");
  int nb = nb_env ? std::atoi(nb_env) : 8;
  nb = std::max(1, std::min(nb, count));
  B->nbranch = nb;
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  auto work = [&](int i) { return (double)B->cls[B->fr[i].cls].elems() * (B->fr[i].N + 0.25); };
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work(x) > work(y); });
  std::vector<double> load(nb, 0.0);
  std::vector<size_t> maxel(nb, 0);
  for (int i : order) {
    const int br = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    B->fr[i].branch = br;
    load[br] += work(i);
    maxel[br] = std::max(maxel[br], B->cls[B->fr[i].cls].elems());
  }
  for (int br = 0; br < nb && s == ILS_OK; ++br) {
    float2 *a = nullptr, *b2 = nullptr;
    if ((e = cudaMalloc((void**)&a, maxel[br] * sizeof(float))) ||
        (e = cudaMalloc((void**)&b2, maxel[br] * sizeof(float)))) {
      cudaFree(a);
      s = e == cudaErrorMemoryAllocation ? ILS_ERR_OOM : fail(e, "cudaMalloc");
      break;
    }
    B->ws.push_back(a);
    B->ws.push_back(b2);
  }
  for (int br = 0; br < nb && s == ILS_OK; ++br) {
    cudaStream_t st;
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking))) { s = fail(e, "cudaStreamCreate"); break; }
    B->streams.push_back(st);
  }
  if (s == ILS_OK && (e = cudaStreamCreateWithFlags(&B->origin, cudaStreamNonBlocking))) s = fail(e, "cudaStreamCreate");
  for (int i = 0; i < nb + 1 && s == ILS_OK; ++i) {
    cudaEvent_t ev;
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming))) { s = fail(e, "cudaEventCreate"); break; }
    B->events.push_back(ev);
  }
  if (s == ILS_OK) s = capture(B);
  if (s != ILS_OK) { release(B); return s; }
  *out = B;
  return ILS_OK;
}

ils_status ils_batch_run(ils_batch* b, void* stream) {
  if (b == nullptr || b->exec == nullptr) return ILS_ERR_INVALID_ARG;
  cudaError_t e = cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? ILS_OK : fail(e, "cudaGraphLaunch");
}

ils_status ils_batch_destroy(ils_batch* b) {
  if (b == nullptr) return ILS_OK;
  cudaError_t e = cudaDeviceSynchronize();
  release(b);
  return e == cudaSuccess ? ILS_OK : fail(e, "cudaDeviceSynchronize");
}

int ils_batch_kernel_choice(const ils_batch* b, int frame, int* row_variant, int* col_variant) {
  if (b == nullptr || frame < 0 || frame >= (int)b->fr.size()) return -1;
  const BatchClass& c = b->cls[b->fr[frame].cls];
  if (row_variant) *row_variant = c.geo.warp_row >= 0 ? 1000 + c.geo.warp_row : c.geo.fixed_row;
  if (col_variant) *col_variant = c.geo.fixed_col;
  return b->fr[frame].branch;
}

ils_status ils_smooth_batched(const ils_frame* frames, int count, void* stream) {
  ils_batch* b = nullptr;
  ils_status s = ils_batch_create(frames, count, 0, &b);
  if (s != ILS_OK) return s;
  s = ils_batch_run(b, stream);
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  ils_status d = ils_batch_destroy(b);
  if (s != ILS_OK) return s;
  if (e != cudaSuccess) return fail(e, "cudaStreamSynchronize");
  return d;
}

}  // extern "C"
