// Warm-started ILS (not in the paper): u^0 = f + net(f) from the warm-start network, then
// a few ILS iterations (Algorithm 1 from u^0 instead of f), with plain ILS from f as the
// fallback when the last iterate change max|u^k - u^{k-1}| exceeds a threshold tau.
#include <cuda_runtime.h>

#include <cstring>
#include <new>

#include "../../include/ils.h"
#include "ils_internal.h"

struct ils_warm {
  ils_plan* warm;   // N = iters, started from u^0
  ils_plan* plain;  // fallback: Algorithm 1 from f
  ils_cnn* net;     // borrowed
  int H, W, C, iters;
  float tau;
  float* u0;        // C x H x W
  float* ckpt;      // iters x C x H x W
  unsigned int* delta_dev;
  unsigned int* delta_host;  // page-locked
  float last_delta;
};

namespace {
void warm_free(ils_warm* w) {
  ils_plan_destroy(w->warm);
  ils_plan_destroy(w->plain);
  cudaFree(w->u0);
  cudaFree(w->ckpt);
  cudaFree(w->delta_dev);
  cudaFreeHost(w->delta_host);
  delete w;
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
  w->H = H; w->W = W; w->C = C; w->iters = iters; w->tau = tau;
  ils_status s;
  if ((s = ils_plan_create(H, W, C, lambda, p, eps, iters, &w->warm)) ||
      (s = ils_plan_create(H, W, C, lambda, p, eps, n_plain, &w->plain))) {
    warm_free(w);
    return s;
  }
  const size_t n = (size_t)C * H * W;
  cudaError_t e;
  if ((e = cudaMalloc((void**)&w->u0, n * 4)) || (e = cudaMalloc((void**)&w->ckpt, n * 4 * iters)) ||
      (e = cudaMalloc((void**)&w->delta_dev, 4)) || (e = cudaMallocHost((void**)&w->delta_host, 4))) {
    warm_free(w);
    ils::record_cuda_error("ils_warm_create", e);
    return e == cudaErrorMemoryAllocation ? ILS_ERR_OOM : ILS_ERR_CUDA;
  }
  *out = w;
  return ILS_OK;
}

ils_status ils_warm_destroy(ils_warm* w) {
  if (w == nullptr) return ILS_OK;
  cudaDeviceSynchronize();
  warm_free(w);
  return ILS_OK;
}

// u = ILS_iters(f; u^0 = f + net(f)), or plain ILS from f if the last change exceeds tau.
// f, u: device C x H x W.  Waits for the change to be known (one 4-byte read).
// *fallback_taken (may be NULL) is set to 1 when the plain path ran; *delta (may be NULL)
// receives the measured change.
ils_status ils_warm_smooth(ils_warm* w, const float* f, float* u, int* fallback_taken, float* delta, void* stream) {
  if (w == nullptr || f == nullptr || u == nullptr) return ILS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t n = (size_t)w->C * w->H * w->W;
  ils_status s;
  if ((s = ils_cnn_infer(w->net, w->C / 3, w->H, w->W, f, w->u0, stream))) return s;
  if ((s = ils_smooth_checkpointed(w->warm, f, w->u0, u, w->ckpt, stream))) return s;
  cudaError_t e;
  if ((e = cudaMemsetAsync(w->delta_dev, 0, 4, st)) ||
      (e = ils::launch_maxabsdiff(u, w->ckpt + (size_t)(w->iters - 1) * n, n, w->delta_dev, st)) ||
      (e = cudaMemcpyAsync(w->delta_host, w->delta_dev, 4, cudaMemcpyDeviceToHost, st)) ||
      (e = cudaStreamSynchronize(st))) {
    ils::record_cuda_error("ils_warm_smooth", e);
    return ILS_ERR_CUDA;
  }
  float d;
  std::memcpy(&d, w->delta_host, 4);
  w->last_delta = d;
  if (delta) *delta = d;
  const bool fb = !(d <= w->tau);
  if (fallback_taken) *fallback_taken = fb ? 1 : 0;
  if (fb) return ils_smooth(w->plain, f, u, stream);
  return ILS_OK;
}

}  // extern "C"
