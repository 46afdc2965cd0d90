// Gaussian pre-smoothing of the input (Sec. 5: texture smoothing pre-smooths the image with a
// small Gaussian before Welsch-penalty ILS).  Separable taps w_k, k = -r..r, periodic wrap
// (the boundary model of Eq. 9's solve); both passes in one kernel on a shared-memory tile.
#include <cuda_runtime.h>

#include <cmath>

namespace ils {
namespace {

constexpr int kBlurTile = 32;
constexpr int kBlurMaxR = 15;  // sigma <= 5 (r = ceil(3 sigma))

struct BlurTaps {
  int r;
  float w[2 * kBlurMaxR + 1];
};

__device__ __forceinline__ int wrap(int i, int n) {
  const int m = i % n;
  return m < 0 ? m + n : m;
}

// One 32 x 32 output tile of channel blockIdx.z: the (32 + 2R)^2 input window (wrapped at
// the image border only) into shared memory, the horizontal pass over all window rows, then
// the vertical pass.  R = the radius, a template parameter so that the tap loops unroll.
template <int R>
__global__ void __launch_bounds__(256) gauss_blur_kernel(const float* __restrict__ in, float* __restrict__ out, int H,
                                                         int W, BlurTaps taps) {
  extern __shared__ float sm[];
  constexpr int T = kBlurTile, E = T + 2 * R;
  float* tin = sm;          // E x E window
  float* th = sm + E * E;   // E x T after the horizontal pass
  const int x0 = blockIdx.x * T, y0 = blockIdx.y * T;
  const size_t plane = (size_t)H * W;
  const float* src = in + blockIdx.z * plane;
  const bool inside = x0 - R >= 0 && y0 - R >= 0 && x0 + T + R <= W && y0 + T + R <= H;
  for (int i = threadIdx.x; i < E * E; i += blockDim.x) {
    const int yy = i / E, xx = i - (i / E) * E;
    const int y = y0 - R + yy, x = x0 - R + xx;
    tin[i] = inside ? src[(size_t)y * W + x] : src[(size_t)wrap(y, H) * W + wrap(x, W)];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < E * T; i += blockDim.x) {
    const int yy = i / T, xx = i - (i / T) * T;
    const float* row = tin + yy * E + xx;
    float acc = 0.0f;
#pragma unroll
    for (int k = 0; k <= 2 * R; ++k) acc = fmaf(taps.w[k], row[k], acc);
    th[i] = acc;
  }
  __syncthreads();
  float* dst = out + blockIdx.z * plane;
  for (int i = threadIdx.x; i < T * T; i += blockDim.x) {
    const int yy = i / T, xx = i - (i / T) * T;
    const int y = y0 + yy, x = x0 + xx;
    if (y >= H || x >= W) continue;
    float acc = 0.0f;
#pragma unroll
    for (int k = 0; k <= 2 * R; ++k) acc = fmaf(taps.w[k], th[(yy + k) * T + xx], acc);
    dst[(size_t)y * W + x] = acc;
  }
}

template <int... Rs>
struct BlurTable {
  static constexpr void (*fns[])(const float*, float*, int, int, BlurTaps) = {gauss_blur_kernel<Rs>...};
};

}  // namespace

// out = the separable periodic Gaussian blur of each H x W channel of f (C channels), taps
// normalized in double precision; 0 <= sigma <= 5, C <= 65535 (checked by the caller).
cudaError_t launch_gaussian_blur(const float* f, float* out, int H, int W, int C, float sigma, cudaStream_t st) {
  BlurTaps taps{};
  taps.r = sigma > 0.0f ? (int)std::ceil(3.0 * (double)sigma) : 0;
  if (taps.r > kBlurMaxR) return cudaErrorInvalidValue;
  double w[2 * kBlurMaxR + 1], sum = 0.0;
  for (int k = -taps.r; k <= taps.r; ++k) {
    w[k + taps.r] = taps.r == 0 ? 1.0 : std::exp(-(double)k * k / (2.0 * (double)sigma * sigma));
    sum += w[k + taps.r];
  }
  for (int k = 0; k <= 2 * taps.r; ++k) taps.w[k] = (float)(w[k] / sum);
  const int E = kBlurTile + 2 * taps.r;
  const size_t smem = (size_t)(E * E + E * kBlurTile) * sizeof(float);
  dim3 grid((W + kBlurTile - 1) / kBlurTile, (H + kBlurTile - 1) / kBlurTile, C);
  using Table = BlurTable<0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15>;
  static_assert(sizeof(Table::fns) / sizeof(Table::fns[0]) == kBlurMaxR + 1, "one kernel per radius");
  Table::fns[taps.r]<<<grid, 256, smem, st>>>(f, out, H, W, taps);
  return cudaGetLastError();
}

}  // namespace ils
