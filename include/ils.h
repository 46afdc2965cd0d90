/*
 * ils.h - C ABI of libils.so: Iterative Least Squares (ILS) edge-preserving
 * smoothing on one NVIDIA GB300 (sm_103a) GPU.
 *
 * Method: Liu, Zhang, Huang, Yang, Shen, Reid, "Real-time Image Smoothing via
 * Iterative Least Squares" (arXiv 2003.07504).  Equation numbers follow the
 * paper's LaTeX order:
 *   Eq. 1  E(u,f) = sum_s (u_s-f_s)^2 + lambda sum_{*=x,y} phi_p(grad_* u_s)      (Sec. 3)
 *   Eq. 2  phi_p(x) = (x^2 + eps)^(p/2)                                          (Sec. 3)
 *   Eq. 7  mu_* = c grad_* u - p grad_* u (grad_* u^2 + eps)^(p/2-1)             (Sec. 3.1)
 *   Eq. 9  u^{n+1} = F^-1[(F f + lambda/2 sum_* conj(F grad_*) F mu_*) /
 *                         (F 1 + c lambda/2 sum_* |F grad_*|^2)]                 (Sec. 3.2)
 *   Eq. 11 c = c0 = p eps^(p/2-1)                                                 (Sec. 3.3, App. B)
 *   Algorithm 1: u^0 = f; N times: mu from u (Eq. 7), u from Eq. 9.
 *   Sec. 3.4: colour channels are smoothed independently.
 *
 * Conventions shared by every entry point
 *   - Images are planar C x H x W float32, row-major, contiguous (x fastest),
 *     caller-owned.  Gradients are periodic forward differences
 *     (grad_x u)[y,x] = u[y,(x+1)%W] - u[y,x], likewise in y (the periodic
 *     boundary that Eq. 9 assumes).
 *   - "Device pointer" means memory the CUDA device can address (cudaMalloc,
 *     torch CUDA tensors).  All calls that take a stream are stream-ordered and
 *     asynchronous: they enqueue work on `stream` (a cudaStream_t; NULL is the
 *     legacy default stream) and return; the caller synchronizes.
 *   - Every call returns an ils_status.  Nothing aborts or throws across the
 *     ABI.  On ILS_ERR_CUDA the text of the CUDA error is available from
 *     ils_last_error() on the calling thread.
 *   - Supported sizes: 2 <= H, W <= 8192, W even, and both H and W of the form
 *     2^a 3^b 5^c (the radices of the hand-written FFT).  Other sizes return
 *     ILS_ERR_UNSUPPORTED_SIZE.
 *   - A plan owns device workspace; it is not safe to use one plan from two
 *     streams or threads at the same time.
 */
#ifndef ILS_H_
#define ILS_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ils_plan ils_plan; /* opaque */

typedef enum {
  ILS_OK = 0,
  ILS_ERR_INVALID_ARG = 1,      /* null pointer, bad parameter, aliasing, wrong state */
  ILS_ERR_UNSUPPORTED_SIZE = 2, /* H or W outside the supported set above */
  ILS_ERR_OOM = 3,              /* a device or host allocation failed */
  ILS_ERR_CUDA = 4,             /* a CUDA runtime call failed; see ils_last_error() */
  ILS_ERR_TIMEOUT = 5,          /* a bounded device-side wait gave up (status word set by a kernel) */
  ILS_ERR_FALLBACK_TAKEN = 6,   /* information, never a call's return value: the warm-started
                                   smoother ran plain ILS instead (ils_warm_smooth's flag) */
} ils_status;

/* Human-readable name of a status code (static storage). */
const char* ils_status_string(ils_status s);

/* Text of the last CUDA error seen by an ILS call on this thread ("" if none). */
const char* ils_last_error(void);

/*
 * ils_plan_create - validate parameters and build a plan for C x H x W images.
 *   lambda >= 0 : smoothing strength (Eq. 1).  lambda = 0 returns f.
 *   0 < p <= 1  : penalty power (Eq. 2; the paper's range, Sec. 3).  p = 2 is
 *                 also accepted: c0 = 2 and mu = 0, i.e. one quadratic solve.
 *   eps > 0     : Charbonnier constant (Eq. 2; the paper fixes 1e-4).
 *   N >= 0      : iterations of Algorithm 1 (the paper fixes 4). N = 0 copies f.
 *   c = c0 = p eps^(p/2-1) (Eq. 11) is used; ils_plan_c() returns it.
 * Allocates device workspace of 2*C*H*W floats plus small tables on the current
 * device.  *out receives the plan (NULL on failure).
 */
ils_status ils_plan_create(int H, int W, int C, float lambda, float p, float eps, int N,
                           ils_plan** out);

/*
 * ils_plan_create_welsch - a plan for ILS with the Welsch penalty (Sec. 5 "Model
 * Extension"): phi_W(x) = 2 gamma^2 (1 - exp(-x^2 / (2 gamma^2))) (Eq. 18), mu update
 * mu = c x - 2 x exp(-x^2 / (2 gamma^2)) (Eq. 19), c = c0 = 2 (Eq. 20, Appendix B).
 * Same passes, layout and entry points as a plan from ils_plan_create (smooth,
 * smooth_from, host, checkpointed, backward); the paper uses it for clip-art artifact
 * removal (lambda = 20-30, gamma = 5/255-10/255, N = 10) and texture smoothing (N = 15).
 *   lambda >= 0, gamma > 0 (finite, 1/(2 gamma^2) finite), N >= 0; shapes as for
 *   ils_plan_create.  Returns ILS_ERR_INVALID_ARG for other parameters.
 */
ils_status ils_plan_create_welsch(int H, int W, int C, float lambda, float gamma, int N, ils_plan** out);

/*
 * ils_plan_create_hqs - the comparison method of Sec. 3.5: half-quadratic splitting
 * (Eq. 12-14) with the L1 penalty phi(x) = |x| (anisotropic total variation).  Iteration n:
 * Q1 mu^n = soft threshold of grad u^n at lambda / (2 beta_n); Q2 u^{n+1} =
 * argmin (u - f)^2 + beta_n (grad u - mu^n)^2, solved by the same FFT passes with the
 * weight beta_n; beta_n = kappa^n beta0.  The paper's Fig. 11 setting: lambda = 0.25,
 * beta0 = 2 lambda, N = 4.
 *   lambda > 0; beta0 > 0, or <= 0 for the paper's 2 lambda; kappa >= 1 (the paper requires
 *   kappa > 1 without a value; 2 is a common choice); N >= 0.
 * Smooth / warm start / host / checkpointed calls work as for any plan; ils_backward returns
 * ILS_ERR_INVALID_ARG (no adjoint of the splitting).
 */
ils_status ils_plan_create_hqs(int H, int W, int C, float lambda, float beta0, float kappa, int N, ils_plan** out);

/* Free a plan and its device memory.  NULL is accepted.  Synchronizes the device. */
ils_status ils_plan_destroy(ils_plan* plan);

/* The constant c the plan uses (Eq. 11).  Returns -1 for NULL. */
float ils_plan_c(const ils_plan* plan);

/*
 * ils_smooth - Algorithm 1 with u^0 = f.
 *   f : device pointer, C x H x W float32 input (read only).
 *   u : device pointer, C x H x W float32 output; must not overlap f.
 *
 * Launch graphs (every smoothing call of a plan): the first call with a given set of
 * pointers (and output-stage parameters) launches its kernels on the stream; the second
 * captures that launch sequence into a CUDA graph on a plan-owned stream, and later calls
 * with the same set replay the graph on the caller's stream - the same kernels, the same
 * bits, the data read at replay time, less launch overhead.  A plan keeps the graphs of its
 * 8 most recently used pointer sets; once it has captured 4 graphs it captures more only
 * while they are replayed at least 4 times per capture (callers that rarely repeat a
 * pointer set keep direct launches).  Not while profiling (ils_set_profiling), for N = 0,
 * or when `stream` is itself being captured (the kernels then join the caller's capture).
 * The environment variable ILS_GRAPHS=0, read once per process, turns it off.
 */
ils_status ils_smooth(ils_plan* plan, const float* f, float* u, void* stream);

/*
 * ils_smooth_enhance - detail enhancement: out = u + k (f - u) with u = ILS(f) (Algorithm 1
 * from u^0 = f), fused into the final inverse row pass (which reads f instead of writing u).
 * k = 0 gives u, k = 1 gives f; the paper's figures boost details with k = 3.
 *   f, out : device pointers, C x H x W float32, non-overlapping.  k finite.
 */
ils_status ils_smooth_enhance(ils_plan* plan, const float* f, float* out, float k, void* stream);

/*
 * ils_smooth_luma - colour option (I) of Sec. 3.4: smooth only the luminance of an RGB
 * image.  Y = 0.299 R + 0.587 G + 0.114 B (BT.601 luma; the paper names no matrix),
 * u_Y = ILS(Y), Y' = u_Y + k (Y - u_Y); the chroma is kept, so every channel changes by
 * Y' - Y:  out_c = rgb_c + (1 - k)(u_Y - Y), in the final inverse row pass.  One channel
 * is smoothed instead of three.
 *   plan : made with C = 1 for the image's H x W (either penalty).
 *   rgb, out : device pointers, 3 x H x W float32 (planar R, G, B), non-overlapping.
 * The first call on a plan allocates an H x W float32 luminance buffer that the plan keeps
 * (make it before any stream capture).  Returns ILS_ERR_INVALID_ARG if C != 1.
 */
ils_status ils_smooth_luma(ils_plan* plan, const float* rgb, float* out, float k, void* stream);

/*
 * ils_smooth_hwc - ils_smooth on pixel-interleaved images (H x W x C float32, the channels of
 * a pixel adjacent, as most image libraries store them).  A gather kernel writes the planar
 * copy that every iteration re-reads (Algorithm 1 re-reads f in each right-hand side) into
 * a plan-owned C x H x W buffer, and the final inverse row pass writes u interleaved, so
 * no planar u is materialised.  Same results as ils_smooth on the transposed image.
 *   f_hwc, u_hwc : device pointers, H x W x C float32, non-overlapping.
 * The first call allocates the planar buffer (C x H x W float32, shared with
 * ils_smooth_host's input staging) that the plan keeps (make it before any stream capture).
 * Returns ILS_ERR_UNSUPPORTED_SIZE when C H W / 2 >= 2^32.
 */
ils_status ils_smooth_hwc(ils_plan* plan, const float* f_hwc, float* u_hwc, void* stream);

/*
 * ils_log_luma - l = ln max(Y, 1e-12) with Y = 0.299 R + 0.587 G + 0.114 B: the logarithm
 * of the luminance on which Sec. 4.2 performs the smoothing for HDR tone mapping (the input
 * of ils_smooth for a base / detail split b = ILS(l), d = l - b).
 *   rgb : device pointer, 3 x H x W float32 (planar R, G, B, linear radiance).
 *   l   : device pointer, H x W float32, not overlapping rgb.
 */
ils_status ils_log_luma(const float* rgb, float* l, int H, int W, void* stream);

/*
 * ils_tonemap_log - single-scale HDR tone mapping of Sec. 4.2: the base layer
 * b = ILS(l) of the log-luminance l (ils_log_luma), detail d = l - b, new log-luminance
 * l' = s b + k d, and the colour ratios kept: out_c = rgb_c exp(l' - l + o)
 *   = rgb_c exp((k - 1) l + (s - k) b + o),
 * written by the final inverse row pass (no b or d is materialised).  s < 1 compresses
 * the base contrast, k > 1 boosts details, o shifts the exposure (log units).  The paper's
 * single-scale setting is p = 1, lambda = 10.
 *   plan : made with C = 1 for the image's H x W.
 *   rgb, out : device pointers, 3 x H x W float32 (planar), non-overlapping.
 * The first call allocates an H x W float32 buffer for l that the plan keeps (shared with
 * ils_smooth_luma).  Returns ILS_ERR_INVALID_ARG if C != 1 or s, k, o are not finite.
 */
ils_status ils_tonemap_log(ils_plan* plan, const float* rgb, float* out, float s, float k, float o, void* stream);

/*
 * ils_gaussian_blur - separable Gaussian blur with periodic wrap: taps w_k, k = -r..r,
 * r = ceil(3 sigma), w_k proportional to exp(-k^2 / (2 sigma^2)) and summing to 1
 * (sigma = 0: a copy).  The pre-smoothing of Sec. 5's texture smoothing.
 *   f, out : device pointers, C x H x W float32, non-overlapping.  0 <= sigma <= 5,
 *            C <= 65535; otherwise ILS_ERR_INVALID_ARG.
 */
ils_status ils_gaussian_blur(const float* f, float* out, int H, int W, int C, float sigma, void* stream);

/*
 * ils_smooth_presmoothed - texture smoothing of Sec. 5: Algorithm 1 on the Gaussian
 * pre-smoothed input (ils_gaussian_blur of f with `sigma`, into a plan-owned buffer; the
 * paper uses a Welsch plan with lambda = 30, gamma = 10/255, N = 15 and a small sigma).
 *   f, u : device pointers, C x H x W float32, non-overlapping.  0 <= sigma <= 5.
 * The first call allocates a C x H x W float32 buffer that the plan keeps (shared with
 * ils_smooth_host's input staging; make it before any stream capture).
 */
ils_status ils_smooth_presmoothed(ils_plan* plan, const float* f, float* u, float sigma, void* stream);

/*
 * ils_smooth_from - Algorithm 1 started from a given u^0 instead of f (warm start).
 *   u0 : device pointer, C x H x W float32 (read only); may equal f.
 *   u  : device pointer output; must overlap neither f nor u0.
 */
ils_status ils_smooth_from(ils_plan* plan, const float* f, const float* u0, float* u, void* stream);

/*
 * ils_smooth_host - ils_smooth on HOST buffers: copies f to the device, runs
 * Algorithm 1, copies u back and synchronizes `stream` before returning.
 *   f_host, u_host : host pointers to C x H x W float32 (page-locked memory
 *                    gives full copy bandwidth; pageable memory also works).
 * Uses device staging buffers owned by the plan (allocated on first use).  With 2-8
 * channels the copies are pipelined per channel group: the groups' input copies run one
 * after another, and each group's kernels and output copy follow its own input copy on its
 * internal stream, so copies overlap the other groups' kernels.  With page-locked buffers
 * the copies are part of the replayed launch graph (see ils_smooth).
 */
ils_status ils_smooth_host(ils_plan* plan, const float* f_host, float* u_host, void* stream);

/*
 * ils_set_checkpointing - plan-owned checkpoints for the adjoint (reverse mode through
 * Algorithm 1; the paper has no adjoint, this is the chain rule through Eq. 9 and Eq. 7).
 *   on != 0 : the plan allocates N x C x H x W float32 (on the current device, once) and every
 *             later ils_smooth / ils_smooth_from call stores its iterates u^0 .. u^{N-1} there
 *             for ils_backward (the same launches, each row pass also writing its u^n).
 *   on == 0 : frees that buffer (synchronizes the device); calls stop storing iterates.
 * Returns ILS_ERR_INVALID_ARG for a half-quadratic-splitting plan (no adjoint), ILS_ERR_OOM
 * if the buffer cannot be allocated.  Allocate before any stream capture.
 */
ils_status ils_set_checkpointing(ils_plan* plan, int on);

/*
 * ils_backward - gradient of a scalar loss L through the plan's last checkpointed smoothing.
 * With A the Eq. 9 operator (symmetric) and g = dL/du^{n+1}, each step n = N-1 .. 0 computes
 * r = A^-1 g with the same FFT solve, adds r to dL/df (the direct dependence through Eq. 9's
 * F(f)), and forms dL/du^n = lambda/2 sum_* grad_*^T [g''(grad_* u^n) * grad_* r], g'' from
 * Appendix B.
 *   f      : the device pointer f of the last ils_smooth / ils_smooth_from call made with
 *            checkpointing on (its checkpoints are used; another pointer, or no such call,
 *            returns ILS_ERR_INVALID_ARG).
 *   grad_u : device pointer, dL/du^N, C x H x W (read only).
 *   grad_f : device pointer, receives dL/df, C x H x W; for ils_smooth (u^0 = f) this
 *            includes the path through u^0, for ils_smooth_from with a separate u^0 only the
 *            direct part (ils_backward_ckpt returns dL/du^0 separately).  Must not overlap
 *            f or grad_u.
 * The first call after a warm-started forward allocates a C x H x W buffer that the plan
 * keeps.  Stream-ordered after the forward on the same stream.
 */
ils_status ils_backward(ils_plan* plan, const float* f, const float* grad_u, float* grad_f, void* stream);

/*
 * ils_smooth_checkpointed - Algorithm 1 (from u0, or from f when u0 is NULL) that
 * also stores the iterates u^0 .. u^{N-1} in a caller-owned buffer for ils_backward_ckpt
 * (for callers that keep several forward results alive at once, e.g. autograd graphs).
 *   ckpt : device pointer, caller-owned, N x C x H x W float32 (iterate n at offset
 *          n*C*H*W); must not overlap f, u0 or u.  May be NULL only when N = 0.
 */
ils_status ils_smooth_checkpointed(ils_plan* plan, const float* f, const float* u0, float* u, float* ckpt,
                                   void* stream);

/*
 * ils_backward_ckpt - ils_backward on caller-owned checkpoints, with the gradient of the
 * starting point available separately.
 *   ckpt    : the iterates written by ils_smooth_checkpointed for this input (read only).
 *   grad_u  : device pointer, dL/du^N, C x H x W (read only).
 *   grad_f  : device pointer, receives dL/df (the direct dependence through Eq. 9's F(f)),
 *             plus dL/du^0 when grad_u0 is NULL (u^0 = f for plain smoothing).
 *   grad_u0 : NULL, or a device pointer receiving dL/du^0 separately (warm starts).
 * Outputs must not overlap each other or grad_u.
 */
ils_status ils_backward_ckpt(ils_plan* plan, const float* ckpt, const float* grad_u, float* grad_f, float* grad_u0,
                             void* stream);

/*
 * Batches of frames of uneven size (not in the paper: a serving-side extension).
 * Each frame carries its own size, parameters and buffers; channels are independent
 * as for a plan.  f and u are device pointers; no frame's u may overlap any frame's f
 * or u, and a frame's f may not overlap its own u.
 */
typedef struct {
  int H, W, C, N;
  float lambda, p, eps;
  const float* f;
  float* u;
} ils_frame;

typedef struct ils_batch ils_batch; /* opaque */

#define ILS_BATCH_AUTOTUNE 1 /* time the kernel variants per size class at creation */

/*
 * ils_batch_create - validate the frames, group them into size classes (shared FFT
 * plans and tables; per-frame Eq. 7 parameters and Eq. 9 denominators), spread them
 * over parallel branches, allocate the workspaces and capture every pass of every
 * frame into one CUDA graph.  The frame pointers are baked into the graph: run the
 * batch only while those buffers are alive, and create a new batch for new buffers.
 * With ILS_BATCH_AUTOTUNE, each size class times its compile-time tile shapes and the
 * generic kernels on the current device and keeps the fastest; if the environment
 * variable ILS_AUTOTUNE_CACHE names a file, choices are read from and appended to it.
 * ILS_BATCH_BRANCHES (default 8) sets the number of parallel branches.
 */
ils_status ils_batch_create(const ils_frame* frames, int count, int flags, ils_batch** out);

/* One graph launch of the whole batch on `stream` (asynchronous). */
ils_status ils_batch_run(ils_batch* batch, void* stream);

/* Free a batch (synchronizes the device).  NULL is accepted. */
ils_status ils_batch_destroy(ils_batch* batch);

/*
 * Introspection for tools and tests: the branch a frame runs on (return value, or -1
 * for a bad argument) and the kernel variants its class uses: row variant 1000 + w for
 * warp-per-row (or warp-pair) kernel entry w, otherwise an index into the table of block-per-strip
 * plans; column variant an index into the table of column plans; -1 = generic kernels.
 */
int ils_batch_kernel_choice(const ils_batch* batch, int frame, int* row_variant, int* col_variant);

/* ils_batch_create (no autotuning) + ils_batch_run + ils_batch_destroy; returns after
 * the batch has finished on `stream`. */
ils_status ils_smooth_batched(const ils_frame* frames, int count, void* stream);

/*
 * Warm-start network (not in the paper): u^0 = f + net(f), net = six 3x3 convolutions
 * 3 -> 32 -> 32 -> 32 -> 32 -> 32 -> 3, ReLU between them, zero padding, BF16 weights
 * and activations with FP32 accumulation on the tensor cores.  Images are batches of
 * B RGB frames: device B x 3 x H x W FP32 planar (the layout of a 3B-channel plan).
 * Parameters, in ils_cnn_set_weights / ils_cnn_get_weights / ils_cnn_get_grads order:
 * for each layer, W[co][ci][ky][kx] then b[co], FP32 host arrays of
 * ils_cnn_param_count() values.
 */
typedef struct ils_cnn ils_cnn; /* opaque: FP32 master weights, BF16 copies, Adam state, activations */

long long ils_cnn_param_count(void);

/* Allocate a network whose forward/backward accept batches of up to max_pixels = B*H*W. */
ils_status ils_cnn_create(long long max_pixels, ils_cnn** out);
ils_status ils_cnn_destroy(ils_cnn* net);                        /* NULL accepted; synchronizes */
ils_status ils_cnn_set_weights(ils_cnn* net, const float* params, long long count);  /* also resets Adam */
ils_status ils_cnn_get_weights(const ils_cnn* net, float* params, long long count);
ils_status ils_cnn_get_grads(const ils_cnn* net, float* grads, long long count);
/* Adam state for training checkpoints: first and second moments in parameter order (host
 * arrays of ils_cnn_param_count() values) and the step count of the bias correction.
 * Restore with ils_cnn_set_adam after ils_cnn_set_weights (which resets the state);
 * step in [0, 2e9]. */
ils_status ils_cnn_get_adam(const ils_cnn* net, float* m, float* v, long long count, long long* step);
ils_status ils_cnn_set_adam(ils_cnn* net, const float* m, const float* v, long long count, long long step);

/* u0 = f + net(f) (f, u0 device, non-overlapping).  Keeps the activations for backward. */
ils_status ils_cnn_forward(ils_cnn* net, int B, int H, int W, const float* f, float* u0, void* stream);

/* u0 = f + net(f) for inference (the last forward's activations are overwritten).  It runs
 * the layer-by-layer kernels of ils_cnn_forward (with tcgen05: 0.40 ms for a 1920 x 1080 RGB
 * frame); with ILS_CNN_FUSED=1 in the environment and the tcgen05 kernels in use, two fused
 * kernels instead, layers 1-3 and 4-6, whose hidden activations stay on chip except the one
 * 32-channel map between them (0.50 ms).  Same numerics either way (BF16 inputs, weights and
 * hidden activations, FP32 accumulation); results agree up to FP32 accumulation order.
 * f, u0: device B x 3 x H x W FP32, non-overlapping. */
ils_status ils_cnn_infer(ils_cnn* net, int B, int H, int W, const float* f, float* u0, void* stream);

/* Accumulate dL/dparams given dL/du0 (device, B x 3 x H x W), using the activations of
 * the last forward call, which must have been on the same f and shape. */
ils_status ils_cnn_backward(ils_cnn* net, int B, int H, int W, const float* f, const float* grad_u0, void* stream);
ils_status ils_cnn_zero_grad(ils_cnn* net, void* stream);

/* Every layer's forward, input gradient and weight gradient runs on the tcgen05 tensor cores
 * (TMA loads, tensor-memory accumulators) when the driver offers tensor-map encoding, else on
 * the mma.sync kernels; ILS_CNN_TC=0 in the environment at creation forces the latter.
 * Returns 1 when the tcgen05 kernels are in use. */
int ils_cnn_uses_tcgen05(const ils_cnn* net);

/* Waits for the device; returns ILS_ERR_TIMEOUT (and clears it) if a tensor-core kernel's
 * bounded wait on its own copies or MMAs gave up since the last check. */
ils_status ils_cnn_check(ils_cnn* net);

/* One Adam step on the FP32 master weights (bias-corrected; the step count is kept in
 * the network), then refresh the BF16 copies. */
ils_status ils_cnn_adam_step(ils_cnn* net, float lr, float beta1, float beta2, float eps, void* stream);

/* grad = 2 (u0 - target) / n and *loss += mean((u0 - target)^2); all device pointers,
 * *loss is FP32 and accumulated (zero it first). */
ils_status ils_mse(const float* u0, const float* target, float* grad, long long n, float* loss, void* stream);

/*
 * Warm-started smoothing: u = ILS_iters(f; u^0 = f + net(f)) (Algorithm 1 from u^0),
 * and plain ILS (n_plain iterations from f) instead when the last iterate change
 * delta = max |u^iters - u^{iters-1}| exceeds tau (a NaN change counts as +inf).
 * C must be a multiple of 3 (RGB frames).  The network is borrowed and must outlive the
 * object.  delta is reduced inside the final inverse row pass and the decision is taken on
 * the device: each call runs as one CUDA graph (network, warm iterations, decision, and a
 * conditional node whose body is the plain ILS), captured at the first call for a given
 * (f, u) pair and replayed for later calls with the same pair.
 */
typedef struct ils_warm ils_warm;
ils_status ils_warm_create(int H, int W, int C, float lambda, float p, float eps, int iters, int n_plain, float tau,
                           ils_cnn* net, ils_warm** out);
ils_status ils_warm_destroy(ils_warm* warm);
/* f, u: device C x H x W, non-overlapping.  With fallback_taken and delta both NULL the call
 * is asynchronous (nothing waits on the host); otherwise it synchronizes `stream` and sets
 * *fallback_taken to ILS_ERR_FALLBACK_TAKEN when the plain path ran (ILS_OK otherwise) and
 * *delta to the warm path's last change.  Returns ILS_ERR_INVALID_ARG when `stream` is being
 * captured (the call launches a graph of its own).  ILS_GRAPHS=0 in the environment keeps
 * direct launches with the decision taken on the host. */
ils_status ils_warm_smooth(ils_warm* warm, const float* f, float* u, int* fallback_taken, float* delta,
                           void* stream);
/* The decision and delta of the last ils_warm_smooth call, once its stream has been
 * synchronized (host arrays written by the call's final device-to-host copy). */
ils_status ils_warm_result(const ils_warm* warm, int* fallback_taken, float* delta);

/*
 * Per-kernel timing, for measurement tools.  Kernel kinds of one ils_smooth call:
 *   ILS_KERNEL_ROW_FIRST   - first fused row pass (reads f or u0; stencil; forward row FFT)
 *   ILS_KERNEL_ROW         - later fused row passes (inverse row FFT of u^n; stencil; forward row FFT)
 *   ILS_KERNEL_COLUMN      - column FFT, Eq. 9 division, inverse column FFT
 *   ILS_KERNEL_ROW_INVERSE - final inverse row FFT writing u^N
 * ils_set_profiling(plan, 1) creates CUDA events and clears the totals; while
 * on, each smoothing call records an event on its stream before every launch
 * and after the last, then waits for its own last event and adds the elapsed
 * times per kind (so profiled calls are synchronous).  ils_set_profiling(plan, 0)
 * turns it off and frees the events.  ils_get_profile copies the totals into
 * ms[ILS_KERNEL_KINDS] and launches[ILS_KERNEL_KINDS] (host arrays).
 */
#define ILS_KERNEL_ROW_FIRST 0
#define ILS_KERNEL_ROW 1
#define ILS_KERNEL_COLUMN 2
#define ILS_KERNEL_ROW_INVERSE 3
#define ILS_KERNEL_KINDS 4
ils_status ils_set_profiling(ils_plan* plan, int on);
ils_status ils_get_profile(const ils_plan* plan, double* ms, long long* launches);

/*
 * ils_smooth_noalloc - ils_smooth for callers that cannot allocate.
 * (The paper has no counterpart; this is a deployment variant of the same path.)
 *
 * Some callers must not allocate once they are running - for example a video
 * pipeline that cannot take cudaMalloc's implicit device synchronization and
 * unbounded latency in the middle of a stream, or a plugin whose host
 * application owns all device memory.  This call runs the same kernels as
 * ils_smooth, but its workspace is a fixed array in the library's static device
 * memory: it calls no cudaMalloc, cudaFree or other allocating routine, host
 * or device.  The caller still passes f and u (device pointers, C x H x W
 * float32, non-overlapping) and a stream; parameters mean what they mean for
 * ils_plan_create, with the same validation.
 *
 * Limits: C*H*W <= ILS_NOALLOC_MAX_ELEMS (2^21 floats, e.g. one 1920 x 1080
 * channel) and H, W <= ILS_NOALLOC_MAX_SIDE; larger images return
 * ILS_ERR_UNSUPPORTED_SIZE.  The array (ILS_NOALLOC_SCRATCH_BYTES = 17,252,608
 * bytes, 16.45 MiB: two image-sized spectra and the largest twiddle and
 * denominator tables) is part of the library: every GPU that loads libils.so
 * holds it until the process exits.
 *
 * A __device__ array has one instance per CUDA context.  The first call in a
 * context (the device's primary context, or a context the host application
 * made current) looks up the array's address in that context and sets the
 * kernels' shared-memory limits there; the result is cached per context (keyed
 * by the context's process-unique identifier, so a context re-created after
 * cudaDeviceReset is set up again).  Make that first call before any stream
 * capture.  All calls in a context share the one array, which keeps the
 * previous call's contents (nothing in it needs to start at zero: every word is
 * written before it is read).  Calls that overlap on the GPU - on two streams,
 * or from two threads - race on it and must be serialized by the caller.
 * Returns ILS_ERR_CUDA if a launch fails.
 */
#define ILS_NOALLOC_MAX_ELEMS (1 << 21)
#define ILS_NOALLOC_MAX_SIDE 8192
#define ILS_NOALLOC_SCRATCH_BYTES 17252608
ils_status ils_smooth_noalloc(int H, int W, int C, float lambda, float p, float eps, int N,
                              const float* f, float* u, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* ILS_H_ */
