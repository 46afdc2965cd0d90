// Warm-started ILS (not in the paper): u^0 = f + net(f) from the warm-start network, then
// a few ILS iterations (Algorithm 1 from u^0 instead of f), with plain ILS from f as the
// fallback when the last iterate change delta = max|u^k - u^{k-1}| exceeds a threshold tau.
//
// delta is reduced in the output stage of the final inverse row pass (output mode 5), which
// writes u^k and compares it with u^{k-1} (u^0 itself for one iteration, else the last
// checkpoint) without another pass over the image.  The decision is taken on the device: a
// call is one CUDA graph - network, warm iterations, a one-thread kernel that sets a
// conditional handle from delta, and an IF node whose body is the plain ILS - so the host
// never waits for delta.  A small device-to-host copy at the end of the graph leaves delta
// and the decision in page-locked memory for ils_warm_result.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>

#include "../../include/ils.h"
#include "ils_internal.h"

namespace ils {
int run_plan_epilogue(ils_plan* pl, const float* f, const float* u0, float* u, float* ckpt, const Epilogue& epi,
                      cudaStream_t st);
}

struct ils_warm {
  ils_plan* warm;   // N = iters, started from u^0
  ils_plan* plain;  // fallback: Algorithm 1 from f
  ils_cnn* net;     // borrowed
  int H, W, C, iters, n_plain;
  float tau;
  float* u0;        // C x H x W
  float* ckpt;      // iters x C x H x W (iters >= 2: the last iterate before u^k)
  unsigned int* words_dev;   // [0] delta (bits of a non-negative float), [1] decision
  unsigned int* words_host;  // page-locked copy written at the end of each call
  // the graph of one call, for the f and u it was captured with
  cudaGraphExec_t exec;
  const float* exec_f;
  float* exec_u;
  cudaStream_t cap;
  bool graph_failed;
};

namespace {

// Sets the conditional handle of the call's graph: run the plain-ILS body when delta > tau
// (a NaN change was recorded as +inf, so it falls back too).
__global__ void warm_decide_kernel(cudaGraphConditionalHandle h, unsigned int* words, float tau) {
  const float d = __uint_as_float(words[0]);
  const bool fb = !(d <= tau);
  words[1] = fb ? (unsigned int)ILS_ERR_FALLBACK_TAKEN : 0u;
  cudaGraphSetConditional(h, fb ? 1u : 0u);
}

void warm_free(ils_warm* w) {
  if (w->exec != nullptr) cudaGraphExecDestroy(w->exec);
  if (w->cap != nullptr) cudaStreamDestroy(w->cap);
  ils_plan_destroy(w->warm);
  ils_plan_destroy(w->plain);
  cudaFree(w->u0);
  cudaFree(w->ckpt);
  cudaFree(w->words_dev);
  cudaFreeHost(w->words_host);
  delete w;
}

bool graphs_on() {
  static const bool on = [] {
    const char* e = std::getenv("ILS_GRAPHS");
    return !(e != nullptr && e[0] == '0');
  }();
  return on;
}

// The warm part of a call on `st`: delta reset, network, iterations with the delta stage.
ils_status enqueue_warm(ils_warm* w, const float* f, float* u, cudaStream_t st) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(w->words_dev, 0, 2 * sizeof(unsigned int), st))) {
    ils::record_cuda_error("ils_warm_smooth", e);
    return ILS_ERR_CUDA;
  }
  ils_status s;
  if ((s = ils_cnn_infer(w->net, w->C / 3, w->H, w->W, f, w->u0, st))) return s;
  ils::Epilogue epi;
  epi.mode = 5;
  const size_t n = (size_t)w->C * w->H * w->W;
  epi.prev = w->iters == 1 ? w->u0 : w->ckpt + (size_t)(w->iters - 1) * n;
  epi.dmax = w->words_dev;
  return (ils_status)ils::run_plan_epilogue(w->warm, f, w->u0, u, w->iters == 1 ? nullptr : w->ckpt, epi, st);
}

// Captures the whole call for (f, u): warm part, decision, IF node with the plain ILS as its
// body, copy of delta and the decision to the host.  Null on any failure.
cudaGraphExec_t capture_call(ils_warm* w, const float* f, float* u) {
  if (w->cap == nullptr && cudaStreamCreateWithFlags(&w->cap, cudaStreamNonBlocking) != cudaSuccess) {
    w->cap = nullptr;
    return nullptr;
  }
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphConditionalHandle h;
  bool ok = cudaGraphCreate(&g, 0) == cudaSuccess &&
            cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault) == cudaSuccess;
  if (ok && cudaStreamBeginCaptureToGraph(w->cap, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
                cudaSuccess) {
    ok = enqueue_warm(w, f, u, w->cap) == ILS_OK;
    if (ok) {
      warm_decide_kernel<<<1, 1, 0, w->cap>>>(h, w->words_dev, w->tau);
      ok = cudaGetLastError() == cudaSuccess;
    }
    cudaGraphNode_t cond = nullptr;
    cudaGraph_t body = nullptr;
    if (ok) {
      cudaStreamCaptureStatus cs;
      cudaGraph_t cg = nullptr;
      const cudaGraphNode_t* deps = nullptr;
      const cudaGraphEdgeData* edges = nullptr;
      size_t nd = 0;
      ok = cudaStreamGetCaptureInfo(w->cap, &cs, nullptr, &cg, &deps, &edges, &nd) == cudaSuccess &&
           cs == cudaStreamCaptureStatusActive;
      if (ok) {
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeIf;
        cp.conditional.size = 1;
        ok = cudaGraphAddNode(&cond, cg, deps, edges, nd, &cp) == cudaSuccess;
        if (ok) body = cp.conditional.phGraph_out[0];
      }
      ok = ok && cudaStreamUpdateCaptureDependencies(w->cap, &cond, nullptr, 1, cudaStreamSetCaptureDependencies) ==
                     cudaSuccess;
    }
    ok = ok && cudaMemcpyAsync(w->words_host, w->words_dev, 2 * sizeof(unsigned int), cudaMemcpyDeviceToHost,
                               w->cap) == cudaSuccess;
    cudaGraph_t out = nullptr;
    ok = cudaStreamEndCapture(w->cap, &out) == cudaSuccess && ok;
    // the fallback body: plain ILS from f into u
    if (ok && cudaStreamBeginCaptureToGraph(w->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
                  cudaSuccess) {
      ok = ils_smooth(w->plain, f, u, w->cap) == ILS_OK;
      cudaGraph_t b2 = nullptr;
      ok = cudaStreamEndCapture(w->cap, &b2) == cudaSuccess && ok;
    } else {
      ok = false;
    }
  } else {
    ok = false;
  }
  if (ok && cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) exec = nullptr;
  if (!ok) exec = nullptr;
  if (g != nullptr) cudaGraphDestroy(g);
  cudaGetLastError();  // a failed capture leaves no sticky error; clear the last one
  return exec;
}

}  // namespace

extern "C" {

ils_status ils_warm_create(int H, int W, int C, float lambda, float p, float eps, int iters, int n_plain, float tau,
                           ils_cnn* net, ils_warm** out) {
  if (out == nullptr || net == nullptr || iters < 1 || n_plain < 0 || C % 3 != 0 || !(tau >= 0.0f))
    return ILS_ERR_INVALID_ARG;
  *out = nullptr;
  ils_warm* w = new (std::nothrow) ils_warm();
  if (w == nullptr) return ILS_ERR_OOM;
  w->net = net;
  w->H = H; w->W = W; w->C = C; w->iters = iters; w->n_plain = n_plain; w->tau = tau;
  ils_status s;
  if ((s = ils_plan_create(H, W, C, lambda, p, eps, iters, &w->warm)) ||
      (s = ils_plan_create(H, W, C, lambda, p, eps, n_plain, &w->plain))) {
    warm_free(w);
    return s;
  }
  const size_t n = (size_t)C * H * W;
  cudaError_t e;
  if ((e = cudaMalloc((void**)&w->u0, n * 4)) ||
      (iters > 1 && (e = cudaMalloc((void**)&w->ckpt, n * 4 * iters))) ||
      (e = cudaMalloc((void**)&w->words_dev, 2 * sizeof(unsigned int))) ||
      (e = cudaMallocHost((void**)&w->words_host, 2 * sizeof(unsigned int)))) {
    warm_free(w);
    ils::record_cuda_error("ils_warm_create", e);
    return e == cudaErrorMemoryAllocation ? ILS_ERR_OOM : ILS_ERR_CUDA;
  }
  std::memset(w->words_host, 0, 2 * sizeof(unsigned int));
  *out = w;
  return ILS_OK;
}

ils_status ils_warm_destroy(ils_warm* w) {
  if (w == nullptr) return ILS_OK;
  cudaDeviceSynchronize();
  warm_free(w);
  return ILS_OK;
}

ils_status ils_warm_result(const ils_warm* w, int* fallback_taken, float* delta) {
  if (w == nullptr) return ILS_ERR_INVALID_ARG;
  unsigned int words[2];
  std::memcpy(words, w->words_host, sizeof(words));
  if (fallback_taken) *fallback_taken = words[1] != 0 ? (int)ILS_ERR_FALLBACK_TAKEN : (int)ILS_OK;
  if (delta) std::memcpy(delta, &words[0], sizeof(float));
  return ILS_OK;
}

ils_status ils_warm_smooth(ils_warm* w, const float* f, float* u, int* fallback_taken, float* delta, void* stream) {
  if (w == nullptr || f == nullptr || u == nullptr) return ILS_ERR_INVALID_ARG;
  const size_t bytes = (size_t)w->C * w->H * w->W * sizeof(float);
  const uintptr_t a = reinterpret_cast<uintptr_t>(f), b = reinterpret_cast<uintptr_t>(u);
  if (a < b + bytes && b < a + bytes) return ILS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return ILS_ERR_INVALID_ARG;
  cudaError_t e;
  if (graphs_on() && !w->graph_failed) {
    if (w->exec == nullptr || w->exec_f != f || w->exec_u != u) {
      if (w->exec != nullptr) {
        cudaGraphExecDestroy(w->exec);
        w->exec = nullptr;
      }
      w->exec = capture_call(w, f, u);
      w->exec_f = f;
      w->exec_u = u;
      w->graph_failed = w->exec == nullptr;
    }
    if (w->exec != nullptr) {
      if ((e = cudaGraphLaunch(w->exec, st))) {
        ils::record_cuda_error("ils_warm_smooth graph launch", e);
        return ILS_ERR_CUDA;
      }
      if (fallback_taken == nullptr && delta == nullptr) return ILS_OK;
      if ((e = cudaStreamSynchronize(st))) {
        ils::record_cuda_error("ils_warm_smooth", e);
        return ILS_ERR_CUDA;
      }
      return ils_warm_result(w, fallback_taken, delta);
    }
  }
  // without graphs: the same warm part, then the decision on the host
  ils_status s;
  if ((s = enqueue_warm(w, f, u, st))) return s;
  if ((e = cudaMemcpyAsync(w->words_host, w->words_dev, sizeof(unsigned int), cudaMemcpyDeviceToHost, st)) ||
      (e = cudaStreamSynchronize(st))) {
    ils::record_cuda_error("ils_warm_smooth", e);
    return ILS_ERR_CUDA;
  }
  float d;
  std::memcpy(&d, w->words_host, sizeof(float));
  const bool fb = !(d <= w->tau);
  w->words_host[1] = fb ? (unsigned int)ILS_ERR_FALLBACK_TAKEN : 0u;
  if (fb && (s = ils_smooth(w->plain, f, u, stream))) return s;
  if (fb && (fallback_taken != nullptr || delta != nullptr) && (e = cudaStreamSynchronize(st))) {
    ils::record_cuda_error("ils_warm_smooth", e);
    return ILS_ERR_CUDA;
  }
  return ils_warm_result(w, fallback_taken, delta);
}

}  // extern "C"
