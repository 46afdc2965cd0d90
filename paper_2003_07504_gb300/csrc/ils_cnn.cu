// Warm-start network for ILS (not in the paper): u0 = f + net(f), net = six 3x3
// convolutions 3->32->32->32->32->32->3 with ReLU between them, BF16 weights and
// activations, FP32 accumulation, on the tensor cores.
//
// Every convolution is an implicit GEMM with M = pixels, N = output channels,
// K = 9 taps x input channels.  A CTA computes an 8 x 16 pixel tile (8 warps, one
// 16-pixel row segment each) with mma.sync m16n8k16 BF16 -> FP32.  The input tile
// (plus a one-pixel halo, zero outside the image) is staged once in shared memory in
// pixel-major order (80-byte pixel stride, conflict free for ldmatrix); the A fragment
// of tap (dy, dx) is an ldmatrix whose row addresses are the shifted pixels, so the
// im2col costs nothing and each input pixel is read from L2 once per layer.  The
// 3-channel planar inputs (the image, or the gradient of the last layer) are unrolled
// into 27 (+5 zero) columns per pixel instead.
//
// Backward: the input gradient of a convolution is the same kernel run with the weights
// flipped in space and transposed in channels (kernels dgrad_*); the weight gradient is
// a GEMM over pixels (dW = sum_p dY(p)^T im2col(X)(p)) computed with the same MMA and
// reduced into FP32 with atomics.  ReLU masks use the stored post-ReLU activations.
// With tcgen05 available, every layer's forward, input gradient and weight gradient runs on
// the tcgen05 kernels of ils_cnn_tc.cu (a 3-channel side packed into NHWC rows first); these
// kernels remain as the whole network without tcgen05 (ILS_CNN_TC=0), the reference the
// tensor-core kernels are tested against.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "../../include/ils.h"
#include "ils_internal.h"

namespace ils {
namespace cnn {

constexpr int TH = 8, TW = 16, NTHREADS = 256;
constexpr int PXS = 40;                       // bf16 per staged pixel (32 + 8 pad: 80 B)
constexpr int HALO_PX = (TH + 2) * (TW + 2);  // 180
constexpr int C = 32;                         // hidden channels
constexpr int KMID = 9 * C;                   // 288
constexpr int KMID_S = KMID + 8;              // smem row stride of weights (bf16)
constexpr int KIN = 32;                       // 27 unrolled taps x 3 channels, padded
constexpr int KIN_S = KIN + 8;

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2(uint32_t addr, uint32_t& r0, uint32_t& r1) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2_t(uint32_t addr, uint32_t& r0, uint32_t& r1) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(addr));
}
// D += A(16x16, row) * B(16x8, col), bf16 in, fp32 accumulate
__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

struct ConvArgs {
  int B, H, W;
  const float* in_planar;  // 3-channel planar FP32 input (B x 3 x H x W), or null
  const bf16* in_nhwc;     // 32-channel NHWC BF16 input, or null
  const bf16* wt;          // [NT*8][K] BF16 weights (K = 288 or 32), rows = output channels
  const float* bias;       // [cout] or null
  bf16* out_nhwc;          // 32-channel NHWC BF16 output
  float* out_planar;       // 3-channel planar FP32 output
  const float* resid;      // added to the planar output (u0 = f + net(f)), or null
  const bf16* mask;        // NHWC BF16; output zeroed where mask <= 0 (ReLU backward), or null
  int relu;                // apply ReLU to the NHWC output
  int cout;                // real output channels
};

// Stage the A source of one tile: the halo tile of a 32-channel NHWC input, or the
// unrolled 3x3x3 neighbourhoods of a 3-channel planar input.
template <bool PLANAR_IN>
__device__ __forceinline__ void stage_input(const ConvArgs& a, bf16* sA, int b, int y0, int x0) {
  const int H = a.H, W = a.W;
  if (!PLANAR_IN) {
    // 180 pixels x 4 chunks of 16 bytes
    const uint4* src = reinterpret_cast<const uint4*>(a.in_nhwc);
    for (int q = threadIdx.x; q < HALO_PX * 4; q += NTHREADS) {
      const int px = q >> 2, ch = q & 3;
      const int hy = px / (TW + 2), hx = px - hy * (TW + 2);
      const int y = y0 - 1 + hy, x = x0 - 1 + hx;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (y >= 0 && y < H && x >= 0 && x < W) v = src[(((size_t)b * H + y) * W + x) * 4 + ch];
      *reinterpret_cast<uint4*>(sA + px * PXS + ch * 8) = v;
    }
  } else {
    // the 3-channel halo tile as FP32 (coalesced along x), then 128 pixels x 32 columns:
    // column k = tap * 3 + c (k < 27), zero beyond
    float* halo = reinterpret_cast<float*>(sA + TH * TW * PXS);   // [3][TH+2][TW+2]
    for (int q = threadIdx.x; q < 3 * HALO_PX; q += NTHREADS) {
      const int c = q / HALO_PX, r = q - c * HALO_PX;
      const int hy = r / (TW + 2), hx = r - hy * (TW + 2);
      const int y = y0 - 1 + hy, x = x0 - 1 + hx;
      float v = 0.0f;
      if (y >= 0 && y < H && x >= 0 && x < W) v = a.in_planar[(((size_t)b * 3 + c) * H + y) * W + x];
      halo[q] = v;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < TH * TW * KIN; q += NTHREADS) {
      const int px = q >> 5, k = q & 31;
      const int ty = px / TW, tx = px - ty * TW;
      float v = 0.0f;
      if (k < 27) {
        const int tap = k / 3, c = k - tap * 3;
        v = halo[c * HALO_PX + (ty + tap / 3) * (TW + 2) + tx + tap % 3];
      }
      sA[px * PXS + k] = __float2bfloat16_rn(v);
    }
  }
}

// out = conv3x3(in) (+bias) (ReLU | mask) (+resid): NT n-tiles of 8 output channels.
template <bool PLANAR_IN, int NT, bool PLANAR_OUT>
__global__ void __launch_bounds__(NTHREADS) conv_fwd_kernel(ConvArgs a) {
  constexpr int K = PLANAR_IN ? KIN : KMID;
  constexpr int KS = PLANAR_IN ? KIN_S : KMID_S;
  extern __shared__ __align__(16) unsigned char smraw[];
  bf16* sW = reinterpret_cast<bf16*>(smraw);            // [NT*8][KS]
  bf16* sA = sW + NT * 8 * KS;                          // halo or unrolled tile
  const int b = blockIdx.z, y0 = blockIdx.y * TH, x0 = blockIdx.x * TW;
  // weights: rows of K bf16 (16-byte chunks)
  for (int q = threadIdx.x; q < NT * 8 * (K / 8); q += NTHREADS) {
    const int r = q / (K / 8), ch = q - r * (K / 8);
    *reinterpret_cast<uint4*>(sW + r * KS + ch * 8) = reinterpret_cast<const uint4*>(a.wt)[r * (K / 8) + ch];
  }
  stage_input<PLANAR_IN>(a, sA, b, y0, x0);
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float acc[NT][4];
#pragma unroll
  for (int n = 0; n < NT; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.0f;
  const int arow = lane & 15, akh = lane >> 4;           // A: row (pixel) and k-half of this lane's address
  const int brow = lane & 7, bkh = (lane >> 3) & 1;      // B: row (out channel) and k-half
  if (!PLANAR_IN) {
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int dy = tap / 3, dx = tap % 3;
      const bf16* arow_p = sA + ((warp + dy) * (TW + 2) + arow + dx) * PXS + akh * 8;
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
        uint32_t a0, a1, a2, a3;
        ldsm_x4(smem_u32(arow_p + kk * 16), a0, a1, a2, a3);
#pragma unroll
        for (int n = 0; n < NT; ++n) {
          uint32_t b0, b1;
          ldsm_x2(smem_u32(sW + (n * 8 + brow) * KS + tap * C + kk * 16 + bkh * 8), b0, b1);
          mma_bf16(acc[n], a0, a1, a2, a3, b0, b1);
        }
      }
    }
  } else {
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
      uint32_t a0, a1, a2, a3;
      ldsm_x4(smem_u32(sA + (warp * TW + arow) * PXS + kk * 16 + akh * 8), a0, a1, a2, a3);
#pragma unroll
      for (int n = 0; n < NT; ++n) {
        uint32_t b0, b1;
        ldsm_x2(smem_u32(sW + (n * 8 + brow) * KS + kk * 16 + bkh * 8), b0, b1);
        mma_bf16(acc[n], a0, a1, a2, a3, b0, b1);
      }
    }
  }

  // epilogue: acc[n][0..1] = pixel g, channels 2t, 2t+1; acc[n][2..3] = pixel g+8
  const int g = lane >> 2, t = lane & 3;
  const int y = y0 + warp;
  if (y >= a.H) return;
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const int x = x0 + g + 8 * half;
    if (x >= a.W) continue;
    const size_t pix = ((size_t)b * a.H + y) * a.W + x;
#pragma unroll
    for (int n = 0; n < NT; ++n) {
      const int co = n * 8 + 2 * t;
      float v0 = acc[n][2 * half], v1 = acc[n][2 * half + 1];
      if (a.bias != nullptr) {
        if (co < a.cout) v0 += a.bias[co];
        if (co + 1 < a.cout) v1 += a.bias[co + 1];
      }
      if (!PLANAR_OUT) {
        if (a.relu) {
          v0 = fmaxf(v0, 0.0f);
          v1 = fmaxf(v1, 0.0f);
        }
        if (a.mask != nullptr) {
          const __nv_bfloat162 m = *reinterpret_cast<const __nv_bfloat162*>(a.mask + pix * C + co);
          if (!(__bfloat162float(m.x) > 0.0f)) v0 = 0.0f;
          if (!(__bfloat162float(m.y) > 0.0f)) v1 = 0.0f;
        }
        *reinterpret_cast<__nv_bfloat162*>(a.out_nhwc + pix * C + co) = __floats2bfloat162_rn(v0, v1);
      } else {
        const size_t hw = (size_t)a.H * a.W, off = (size_t)y * a.W + x;
        if (co < a.cout) {
          const size_t o = ((size_t)b * 3 + co) * hw + off;
          a.out_planar[o] = v0 + (a.resid ? a.resid[o] : 0.0f);
        }
        if (co + 1 < a.cout) {
          const size_t o = ((size_t)b * 3 + co + 1) * hw + off;
          a.out_planar[o] = v1 + (a.resid ? a.resid[o] : 0.0f);
        }
      }
    }
  }
}

// ---------------------------------------------------------------- weight gradient
// dW[co][k] += sum_p dY[p][co] * X_unrolled[p][k], db[co] += sum_p dY[p][co]:
// a GEMM with M = output channels (MT tiles of 16), N = k (8-wide tiles), K = pixels.
// dY is staged [pixel][co] (NHWC BF16, or 3-channel planar FP32 converted), the input
// as for the forward kernel; ldmatrix.trans turns both into the fragments.  Each CTA
// sweeps several pixel tiles, then adds its partial sums into FP32 dW with atomics.
struct WgradArgs {
  int B, H, W;
  const bf16* dy_nhwc;      // 32-channel gradient (NHWC BF16), or null
  const float* dy_planar;   // 3-channel gradient (planar FP32), or null
  const bf16* in_nhwc;      // layer input, 32-channel NHWC
  const float* in_planar;   // layer input, 3-channel planar
  float* dw;                // [cout][K] FP32 (accumulated)
  float* db;                // [cout] FP32 (accumulated)
  int cout;
  int tiles_x, tiles_y;
};

template <bool PLANAR_IN, bool PLANAR_DY>
__global__ void __launch_bounds__(NTHREADS) conv_wgrad_kernel(WgradArgs a) {
  constexpr int K = PLANAR_IN ? KIN : KMID;        // columns of dW
  constexpr int NKT = K / 8;                         // n-tiles (36 or 4)
  constexpr int MT = PLANAR_DY ? 1 : 2;              // 16-row tiles of output channels
  constexpr int DYS = 40;                            // bf16 per staged dY pixel (32 + pad)
  constexpr int FRAGS = MT * NKT;                    // (m-tile, n-tile) pairs
  constexpr int PER_WARP = (FRAGS + 7) / 8;
  extern __shared__ __align__(16) unsigned char smraw[];
  bf16* sDY = reinterpret_cast<bf16*>(smraw);        // [128 px][DYS]
  bf16* sA = sDY + TH * TW * DYS;                    // input tile as in the forward kernel
  __shared__ float sdb[32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float acc[PER_WARP][4];
#pragma unroll
  for (int i = 0; i < PER_WARP; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.0f;
  if (threadIdx.x < 32) sdb[threadIdx.x] = 0.0f;
  const int ntiles = a.B * a.tiles_y * a.tiles_x;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int b = tile / (a.tiles_y * a.tiles_x);
    const int r = tile - b * a.tiles_y * a.tiles_x;
    const int y0 = (r / a.tiles_x) * TH, x0 = (r % a.tiles_x) * TW;
    __syncthreads();
    // dY tile [px][co] (zero outside the image; channels beyond cout zero)
    for (int q = threadIdx.x; q < TH * TW * 32; q += NTHREADS) {
      const int px = q >> 5, co = q & 31;
      const int y = y0 + px / TW, x = x0 + px % TW;
      float v = 0.0f;
      if (y < a.H && x < a.W) {
        if (PLANAR_DY) {
          if (co < a.cout) v = a.dy_planar[(((size_t)b * 3 + co) * a.H + y) * a.W + x];
        } else {
          v = __bfloat162float(a.dy_nhwc[(((size_t)b * a.H + y) * a.W + x) * C + co]);
        }
      }
      sDY[px * DYS + co] = __float2bfloat16_rn(v);
    }
    {
      ConvArgs ca{};
      ca.H = a.H; ca.W = a.W; ca.in_nhwc = a.in_nhwc; ca.in_planar = a.in_planar;
      stage_input<PLANAR_IN>(ca, sA, b, y0, x0);
    }
    __syncthreads();
    // bias gradient: column sums of the staged dY
    if (threadIdx.x < 32) {
      float s = 0.0f;
      for (int px = 0; px < TH * TW; ++px) s += __bfloat162float(sDY[px * DYS + threadIdx.x]);
      sdb[threadIdx.x] += s;
    }
    // K = 128 pixels in 8 steps of 16 (one tile row of 16 pixels per step)
#pragma unroll 1
    for (int ks = 0; ks < TH; ++ks) {
#pragma unroll
      for (int i = 0; i < PER_WARP; ++i) {
        const int fi = warp + 8 * i;
        if (fi >= FRAGS) break;
        const int mt = fi / NKT, nt = fi - mt * NKT;
        // A = dY^T (rows co, cols px): trans-load 16 px x 16 co; lane -> pixel row, co half
        uint32_t a0, a1, a2, a3;
        {
          // matrices: (px 0-7, co 0-7), (px 0-7, co 8-15), (px 8-15, co 0-7), (px 8-15, co 8-15)
          // transposed they give A rows co 0-7 / 8-15 and k (px) 0-7 / 8-15 in a0..a3 order:
          // a0: co 0-7, px 0-7; a1: co 8-15, px 0-7; a2: co 0-7, px 8-15; a3: co 8-15, px 8-15
          const int mi = lane >> 3, rr = lane & 7;
          const int px = ks * TW + rr + ((mi >> 1) << 3);
          const int co = mt * 16 + ((mi & 1) << 3);
          ldsm_x4_t(smem_u32(sDY + px * DYS + co), a0, a1, a2, a3);
        }
        // B = X_unrolled (rows px = k-dim, cols k = n-dim): trans-load 16 px x 8 columns
        uint32_t b0, b1;
        {
          const int mi = (lane >> 3) & 1, rr = lane & 7;
          const int pxl = rr + (mi << 3);  // pixel within this 16-pixel row segment
          const bf16* src;
          if (PLANAR_IN) {
            src = sA + (ks * TW + pxl) * PXS + nt * 8;
          } else {
            const int tap = nt / 4, cb = (nt & 3) * 8;  // column k = tap * 32 + ci
            src = sA + ((ks + tap / 3) * (TW + 2) + pxl + tap % 3) * PXS + cb;
          }
          ldsm_x2_t(smem_u32(src), b0, b1);
        }
        mma_bf16(acc[i], a0, a1, a2, a3, b0, b1);
      }
    }
  }
  __syncthreads();
  // accumulate: acc[i][0..1] = (co = mt*16 + g, k = nt*8 + 2t, +1), acc[i][2..3] = co + 8
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int i = 0; i < PER_WARP; ++i) {
    const int fi = warp + 8 * i;
    if (fi >= FRAGS) break;
    const int mt = fi / NKT, nt = fi - mt * NKT;
    const int co0 = mt * 16 + g, k = nt * 8 + 2 * t;
    if (co0 < a.cout) {
      atomicAdd(&a.dw[co0 * K + k], acc[i][0]);
      atomicAdd(&a.dw[co0 * K + k + 1], acc[i][1]);
    }
    if (co0 + 8 < a.cout) {
      atomicAdd(&a.dw[(co0 + 8) * K + k], acc[i][2]);
      atomicAdd(&a.dw[(co0 + 8) * K + k + 1], acc[i][3]);
    }
  }
  if (threadIdx.x < a.cout) atomicAdd(&a.db[threadIdx.x], sdb[threadIdx.x]);
}

// ---------------------------------------------------------------- small helpers

// Every weight array of the network in one launch: job j covers the flat indices
// [start[j], start[j + 1]) (at most kMaxJobs jobs; a thread finds its job by a linear scan).
constexpr int kMaxJobs = 12;

__device__ __forceinline__ int find_job(const int* start, int count, int i) {
  int j = 0;
  while (j + 1 < count && i >= start[j + 1]) ++j;
  return j;
}

struct PackJob {
  const float* w;   // FP32 master weights [co_n][kpad]
  bf16* out;        // [co_pad][kcols] BF16
  int co_n, ci_n, co_pad, kcols, transpose_flip;
};
struct PackSet {
  int count;
  int start[kMaxJobs + 1];
  PackJob job[kMaxJobs];
};

// Master FP32 weights [co][kpad] (column k = tap * ci_n + ci, tap = 3 ky + kx) -> BF16 GEMM
// rows for the forward conv ([co_pad][kcols], rows >= co_n zero) or, with transpose_flip,
// for the input-gradient conv: it maps the co_n-channel gradient to ci_n channels, so row
// r = ci and column k' = tap' * co_n + co read the weight of tap 8 - tap' (the flipped
// kernel).  Every layer's arrays in one launch.
__global__ void pack_all_kernel(PackSet s) {
  const int total = s.start[s.count];
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
    const int j = find_job(s.start, s.count, q);
    const PackJob& pj = s.job[j];
    const int e = q - s.start[j];
    const int kpad = pj.ci_n == 3 ? KIN : KMID;
    const int r = e / pj.kcols, k = e - r * pj.kcols;
    float v = 0.0f;
    if (!pj.transpose_flip) {
      if (r < pj.co_n && k < 9 * pj.ci_n) v = pj.w[r * kpad + k];
    } else {
      const int tapp = k / pj.co_n, co = k - tapp * pj.co_n;
      if (r < pj.ci_n && tapp < 9) v = pj.w[co * kpad + (8 - tapp) * pj.ci_n + r];
    }
    pj.out[e] = __float2bfloat16_rn(v);
  }
}

struct ParamSet {
  int count;
  int start[kMaxJobs + 1];
  float* w[kMaxJobs];
  float* g[kMaxJobs];
  float* m[kMaxJobs];
  float* v[kMaxJobs];
};

// Adam on FP32 master weights: m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
// w -= lr * mhat / (sqrt(vhat) + eps), with bias corrections c1 = 1 - b1^t, c2 = 1 - b2^t
// (every weight and bias array of the network in one launch).
__global__ void adam_all_kernel(ParamSet s, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int total = s.start[s.count];
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
    const int j = find_job(s.start, s.count, q);
    const int i = q - s.start[j];
    const float gi = s.g[j][i];
    const float mi = b1 * s.m[j][i] + (1.0f - b1) * gi;
    const float vi = b2 * s.v[j][i] + (1.0f - b2) * gi * gi;
    s.m[j][i] = mi;
    s.v[j][i] = vi;
    s.w[j][i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// zeroes the gradient arrays g[j] of the set (one launch)
__global__ void zero_all_kernel(ParamSet s) {
  const int total = s.start[s.count];
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
    const int j = find_job(s.start, s.count, q);
    s.g[j][q - s.start[j]] = 0.0f;
  }
}

// grad = 2 (u0 - target) / n_total; loss partial sums of (u0 - target)^2 into *loss
// (16-byte accesses when the three arrays allow them, the remainder element-wise)
__global__ void mse_kernel(const float* u0, const float* target, float* grad, size_t n, float scale,
                           float* loss) {
  float s = 0.0f;
  const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
  size_t done = 0;
  if (((reinterpret_cast<uintptr_t>(u0) | reinterpret_cast<uintptr_t>(target) | reinterpret_cast<uintptr_t>(grad)) &
       15) == 0) {
    const size_t n4 = n / 4;
    const float4* a = reinterpret_cast<const float4*>(u0);
    const float4* b = reinterpret_cast<const float4*>(target);
    float4* g = reinterpret_cast<float4*>(grad);
    for (size_t i = t0; i < n4; i += stride) {
      const float4 x = a[i], y = b[i];
      const float d0 = x.x - y.x, d1 = x.y - y.y, d2 = x.z - y.z, d3 = x.w - y.w;
      g[i] = make_float4(2.0f * d0 * scale, 2.0f * d1 * scale, 2.0f * d2 * scale, 2.0f * d3 * scale);
      s += (d0 * d0 + d1 * d1) + (d2 * d2 + d3 * d3);
    }
    done = n4 * 4;
  }
  for (size_t i = done + t0; i < n; i += stride) {
    const float d = u0[i] - target[i];
    grad[i] = 2.0f * d * scale;
    s += d * d;
  }
  // one atomic per block (one per warp on the single loss word serialized ~30 k atomics)
  __shared__ float ws[32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    float t = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0f;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) atomicAdd(loss, t * scale);
  }
}

}  // namespace cnn
}  // namespace ils

// ================================================================ host side
using namespace ils::cnn;

namespace {

constexpr int kLayers = 6;
constexpr int kCin[kLayers] = {3, 32, 32, 32, 32, 32};
constexpr int kCout[kLayers] = {32, 32, 32, 32, 32, 3};

int kpad(int l) { return kCin[l] == 3 ? KIN : KMID; }            // GEMM columns of layer l
int copad(int l) { return kCout[l] == 3 ? 8 : 32; }              // padded output rows (forward)
int dg_kpad(int l) { return kCout[l] == 3 ? KIN : KMID; }        // columns of the input-gradient conv
size_t param_count() {
  size_t n = 0;
  for (int l = 0; l < kLayers; ++l) n += (size_t)kCout[l] * kCin[l] * 9 + kCout[l];
  return n;
}

// planar inputs: unrolled tile (bf16) followed by the FP32 3-channel halo tile
constexpr int kPlanarA = TH * TW * PXS + 2 * 3 * HALO_PX;   // in bf16 units
size_t conv_smem(bool planar_in, int nt) {
  const int ks = planar_in ? KIN_S : KMID_S;
  const int a = planar_in ? kPlanarA : HALO_PX * PXS;
  return (size_t)(nt * 8 * ks + a) * sizeof(bf16);
}
size_t wgrad_smem(bool planar_in) {
  const int a = planar_in ? kPlanarA : HALO_PX * PXS;
  return (size_t)(TH * TW * 40 + a) * sizeof(bf16);
}

}  // namespace

struct ils_cnn {
  size_t max_px;
  float* w[kLayers];     // FP32 master weights [cout][kpad]
  float* b[kLayers];     // FP32 biases [cout]
  float* gw[kLayers];    // gradients (same layouts)
  float* gb[kLayers];
  float* mw[kLayers];    // Adam moments
  float* vw[kLayers];
  float* mb[kLayers];
  float* vb[kLayers];
  bf16* wf[kLayers];     // forward BF16 weights [copad][kpad]
  bf16* wd[kLayers];     // input-gradient BF16 weights [cin][dg_kpad] (layers 1..5)
  bf16* act[kLayers - 1];  // post-ReLU activations of layers 0..4, NHWC BF16 [max_px][32]
  bf16* gact[2];           // gradient ping-pong, NHWC BF16
  bf16* pk8;               // a 3-channel plane set as NHWC rows of 8 BF16 (dL/du0 in the backward)
  bf16* pkf;               // f as NHWC rows of 8 BF16, written by the forward (layer 0's input)
  // f and dL/du0 as NHWC rows of 32 BF16 whose channels 3-31 stay zero (zeroed once): the
  // weight gradients read whole 64-byte pixels instead of TMA's zero fill of 8-channel rows
  bf16* pk32[2];
  int step;
  bool packed;
  int* err;    // device flag raised by a tensor-core kernel whose bounded wait gave up
  bool tc;     // middle layers on the tcgen05 kernel
};

namespace {

ils_status cnn_fail(cudaError_t e, const char* where) {
  ils::record_cuda_error(where, e);
  return e == cudaErrorMemoryAllocation ? ILS_ERR_OOM : ILS_ERR_CUDA;
}

void cnn_free(ils_cnn* n) {
  for (int l = 0; l < kLayers; ++l) {
    cudaFree(n->w[l]); cudaFree(n->b[l]); cudaFree(n->gw[l]); cudaFree(n->gb[l]);
    cudaFree(n->mw[l]); cudaFree(n->vw[l]); cudaFree(n->mb[l]); cudaFree(n->vb[l]);
    cudaFree(n->wf[l]); cudaFree(n->wd[l]);
  }
  for (int l = 0; l < kLayers - 1; ++l) cudaFree(n->act[l]);
  cudaFree(n->gact[0]);
  cudaFree(n->gact[1]);
  cudaFree(n->pk8);
  cudaFree(n->pkf);
  cudaFree(n->pk32[0]);
  cudaFree(n->pk32[1]);
  cudaFree(n->err);
  delete n;
}

// planar FP32 [B][3][H][W] -> NHWC BF16 rows of 8 channels (3 values, then 5 zeros), the
// layout the tensor-core weight gradient reads a 3-channel side in
__global__ void planar3_to_nhwc8_kernel(const float* __restrict__ in, size_t hw, size_t n_px, bf16* __restrict__ out,
                                        bf16* __restrict__ out32) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n_px; i += (size_t)gridDim.x * blockDim.x) {
    const size_t b = i / hw, r = i - b * hw;
    const float* src = in + b * 3 * hw + r;
    __nv_bfloat162 c01 = __floats2bfloat162_rn(src[0], src[hw]);
    __nv_bfloat162 c2z = __floats2bfloat162_rn(src[2 * hw], 0.0f);
    uint4 v;
    v.x = *reinterpret_cast<uint32_t*>(&c01);
    v.y = *reinterpret_cast<uint32_t*>(&c2z);
    v.z = 0u;
    v.w = 0u;
    if (out != nullptr) reinterpret_cast<uint4*>(out)[i] = v;
    if (out32 != nullptr) reinterpret_cast<uint4*>(out32)[4 * i] = v;  // channels 8-31 stay zero
  }
}

// out (or null): rows of 8 channels; out32 (or null): the same 16 bytes at the start of rows of
// 32 channels whose other 48 bytes are zero
void planar3_to_nhwc8(const float* in, int B, int H, int W, bf16* out, cudaStream_t st, bf16* out32 = nullptr) {
  const size_t hw = (size_t)H * W, n_px = (size_t)B * hw;
  const size_t blocks = (n_px + 255) / 256;
  planar3_to_nhwc8_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(in, hw, n_px, out, out32);
}

cudaError_t cnn_pack(ils_cnn* n, cudaStream_t st) {
  // forward weights of every layer, input-gradient weights of layers 1..5
  PackSet ps{};
  int at = 0;
  auto add = [&](const PackJob& j) {
    ps.start[ps.count] = at;
    ps.job[ps.count++] = j;
    at += j.co_pad * j.kcols;
  };
  for (int l = 0; l < kLayers; ++l) {
    add(PackJob{n->w[l], n->wf[l], kCout[l], kCin[l], copad(l), kpad(l), 0});
    if (l > 0) add(PackJob{n->w[l], n->wd[l], kCout[l], kCin[l], 32, dg_kpad(l), 1});
  }
  ps.start[ps.count] = at;
  pack_all_kernel<<<(at + 255) / 256, 256, 0, st>>>(ps);
  n->packed = true;
  return cudaGetLastError();
}

// the weights and biases of every layer with their gradients and Adam moments
ParamSet cnn_params(ils_cnn* n) {
  ParamSet s{};
  int at = 0;
  for (int l = 0; l < kLayers; ++l) {
    const int sizes[2] = {kCout[l] * kpad(l), kCout[l]};
    float* w[2] = {n->w[l], n->b[l]};
    float* g[2] = {n->gw[l], n->gb[l]};
    float* m[2] = {n->mw[l], n->mb[l]};
    float* v[2] = {n->vw[l], n->vb[l]};
    for (int t = 0; t < 2; ++t) {
      const int j = s.count++;
      s.start[j] = at;
      s.w[j] = w[t]; s.g[j] = g[t]; s.m[j] = m[t]; s.v[j] = v[t];
      at += sizes[t];
    }
  }
  s.start[s.count] = at;
  return s;
}

dim3 tile_grid(int B, int H, int W) { return dim3((W + TW - 1) / TW, (H + TH - 1) / TH, B); }

bool cnn_shape_ok(const ils_cnn* n, int B, int H, int W) {
  return n != nullptr && B >= 1 && H >= 1 && W >= 1 && (size_t)B * H * W <= n->max_px;
}

}  // namespace

extern "C" {

ils_status ils_cnn_create(long long max_pixels, ils_cnn** out) {
  if (out == nullptr || max_pixels < 1) return ILS_ERR_INVALID_ARG;
  *out = nullptr;
  ils_cnn* n = new (std::nothrow) ils_cnn();
  if (n == nullptr) return ILS_ERR_OOM;
  n->max_px = (size_t)max_pixels;
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < kLayers && e == cudaSuccess; ++l) {
    const size_t nw = (size_t)kCout[l] * kpad(l), nb = kCout[l];
    float** f32[] = {&n->w[l], &n->gw[l], &n->mw[l], &n->vw[l]};
    for (float** p : f32)
      if (e == cudaSuccess && (e = cudaMalloc((void**)p, nw * 4)) == cudaSuccess) e = cudaMemset(*p, 0, nw * 4);
    float** f32b[] = {&n->b[l], &n->gb[l], &n->mb[l], &n->vb[l]};
    for (float** p : f32b)
      if (e == cudaSuccess && (e = cudaMalloc((void**)p, nb * 4)) == cudaSuccess) e = cudaMemset(*p, 0, nb * 4);
    if (e == cudaSuccess) e = cudaMalloc((void**)&n->wf[l], (size_t)copad(l) * kpad(l) * sizeof(bf16));
    if (e == cudaSuccess && l > 0) e = cudaMalloc((void**)&n->wd[l], (size_t)32 * dg_kpad(l) * sizeof(bf16));
  }
  for (int l = 0; l < kLayers - 1 && e == cudaSuccess; ++l)
    e = cudaMalloc((void**)&n->act[l], n->max_px * C * sizeof(bf16));
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaMalloc((void**)&n->gact[i], n->max_px * C * sizeof(bf16));
  if (e == cudaSuccess && (e = cudaMalloc((void**)&n->err, sizeof(int))) == cudaSuccess) e = cudaMemset(n->err, 0, 4);
  // ILS_CNN_TC=0 keeps every layer on the mma.sync kernels
  const char* tcenv = getenv("ILS_CNN_TC");
  n->tc = ils::conv32_tc_available() && !(tcenv != nullptr && tcenv[0] == '0');
  if (e == cudaSuccess && n->tc) e = ils::conv32_tc_set_attributes();
  if (e == cudaSuccess && n->tc) e = ils::warm_fused_set_attributes();
  if (e == cudaSuccess && n->tc) e = cudaMalloc((void**)&n->pk8, n->max_px * 8 * sizeof(bf16));
  if (e == cudaSuccess && n->tc) e = cudaMalloc((void**)&n->pkf, n->max_px * 8 * sizeof(bf16));
  for (int i = 0; i < 2 && e == cudaSuccess && n->tc; ++i)
    if ((e = cudaMalloc((void**)&n->pk32[i], n->max_px * 32 * sizeof(bf16))) == cudaSuccess)
      e = cudaMemset(n->pk32[i], 0, n->max_px * 32 * sizeof(bf16));
  if (e == cudaSuccess) {
    cudaFuncSetAttribute(conv_fwd_kernel<false, 4, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)conv_smem(false, 4));
    cudaFuncSetAttribute(conv_fwd_kernel<false, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)conv_smem(false, 1));
    cudaFuncSetAttribute(conv_fwd_kernel<true, 4, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)conv_smem(true, 4));
    cudaFuncSetAttribute(conv_wgrad_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)wgrad_smem(false));
    cudaFuncSetAttribute(conv_wgrad_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)wgrad_smem(false));
    cudaFuncSetAttribute(conv_wgrad_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)wgrad_smem(true));
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    cnn_free(n);
    return cnn_fail(e, "ils_cnn_create");
  }
  n->step = 0;
  n->packed = false;
  *out = n;
  return ILS_OK;
}

ils_status ils_cnn_destroy(ils_cnn* n) {
  if (n == nullptr) return ILS_OK;
  cudaError_t e = cudaDeviceSynchronize();
  cnn_free(n);
  return e == cudaSuccess ? ILS_OK : cnn_fail(e, "cudaDeviceSynchronize");
}

long long ils_cnn_param_count(void) { return (long long)param_count(); }

// params: per layer W[co][ci][3][3] then b[co] (FP32, host)
ils_status ils_cnn_set_weights(ils_cnn* n, const float* params, long long count) {
  if (n == nullptr || params == nullptr || count != (long long)param_count()) return ILS_ERR_INVALID_ARG;
  size_t off = 0;
  cudaError_t e;
  for (int l = 0; l < kLayers; ++l) {
    const int co_n = kCout[l], ci_n = kCin[l], K = kpad(l);
    std::vector<float> w((size_t)co_n * K, 0.0f);
    for (int co = 0; co < co_n; ++co)
      for (int ci = 0; ci < ci_n; ++ci)
        for (int tap = 0; tap < 9; ++tap) w[(size_t)co * K + tap * ci_n + ci] = params[off + ((size_t)co * ci_n + ci) * 9 + tap];
    off += (size_t)co_n * ci_n * 9;
    if ((e = cudaMemcpy(n->w[l], w.data(), w.size() * 4, cudaMemcpyHostToDevice))) return cnn_fail(e, "set_weights");
    if ((e = cudaMemcpy(n->b[l], params + off, (size_t)co_n * 4, cudaMemcpyHostToDevice))) return cnn_fail(e, "set_weights");
    off += co_n;
    cudaMemset(n->mw[l], 0, w.size() * 4);
    cudaMemset(n->vw[l], 0, w.size() * 4);
    cudaMemset(n->mb[l], 0, (size_t)co_n * 4);
    cudaMemset(n->vb[l], 0, (size_t)co_n * 4);
  }
  n->step = 0;
  if ((e = cnn_pack(n, nullptr))) return cnn_fail(e, "pack");
  if ((e = cudaDeviceSynchronize())) return cnn_fail(e, "set_weights");
  return ILS_OK;
}

ils_status ils_cnn_get_weights(const ils_cnn* n, float* params, long long count) {
  if (n == nullptr || params == nullptr || count != (long long)param_count()) return ILS_ERR_INVALID_ARG;
  size_t off = 0;
  cudaError_t e;
  if ((e = cudaDeviceSynchronize())) return cnn_fail(e, "get_weights");
  for (int l = 0; l < kLayers; ++l) {
    const int co_n = kCout[l], ci_n = kCin[l], K = kpad(l);
    std::vector<float> w((size_t)co_n * K);
    if ((e = cudaMemcpy(w.data(), n->w[l], w.size() * 4, cudaMemcpyDeviceToHost))) return cnn_fail(e, "get_weights");
    for (int co = 0; co < co_n; ++co)
      for (int ci = 0; ci < ci_n; ++ci)
        for (int tap = 0; tap < 9; ++tap) params[off + ((size_t)co * ci_n + ci) * 9 + tap] = w[(size_t)co * K + tap * ci_n + ci];
    off += (size_t)co_n * ci_n * 9;
    if ((e = cudaMemcpy(params + off, n->b[l], (size_t)co_n * 4, cudaMemcpyDeviceToHost))) return cnn_fail(e, "get_weights");
    off += co_n;
  }
  return ILS_OK;
}

// Adam state (first and second moments, in parameter order, and the step count): the
// checkpoint of a training run, restored after ils_cnn_set_weights (which resets it).
ils_status ils_cnn_get_adam(const ils_cnn* n, float* m, float* v, long long count, long long* step) {
  if (n == nullptr || m == nullptr || v == nullptr || step == nullptr || count != (long long)param_count())
    return ILS_ERR_INVALID_ARG;
  cudaError_t e;
  if ((e = cudaDeviceSynchronize())) return cnn_fail(e, "get_adam");
  for (int which = 0; which < 2; ++which) {
    float* dst = which == 0 ? m : v;
    size_t off = 0;
    for (int l = 0; l < kLayers; ++l) {
      const int co_n = kCout[l], ci_n = kCin[l], K = kpad(l);
      std::vector<float> w((size_t)co_n * K);
      if ((e = cudaMemcpy(w.data(), which == 0 ? n->mw[l] : n->vw[l], w.size() * 4, cudaMemcpyDeviceToHost)))
        return cnn_fail(e, "get_adam");
      for (int co = 0; co < co_n; ++co)
        for (int ci = 0; ci < ci_n; ++ci)
          for (int tap = 0; tap < 9; ++tap) dst[off + ((size_t)co * ci_n + ci) * 9 + tap] = w[(size_t)co * K + tap * ci_n + ci];
      off += (size_t)co_n * ci_n * 9;
      if ((e = cudaMemcpy(dst + off, which == 0 ? n->mb[l] : n->vb[l], (size_t)co_n * 4, cudaMemcpyDeviceToHost)))
        return cnn_fail(e, "get_adam");
      off += co_n;
    }
  }
  *step = n->step;
  return ILS_OK;
}

ils_status ils_cnn_set_adam(ils_cnn* n, const float* m, const float* v, long long count, long long step) {
  if (n == nullptr || m == nullptr || v == nullptr || count != (long long)param_count() || step < 0 ||
      step > 2000000000LL)
    return ILS_ERR_INVALID_ARG;
  cudaError_t e;
  for (int which = 0; which < 2; ++which) {
    const float* src = which == 0 ? m : v;
    size_t off = 0;
    for (int l = 0; l < kLayers; ++l) {
      const int co_n = kCout[l], ci_n = kCin[l], K = kpad(l);
      std::vector<float> w((size_t)co_n * K, 0.0f);   // padding columns stay zero
      for (int co = 0; co < co_n; ++co)
        for (int ci = 0; ci < ci_n; ++ci)
          for (int tap = 0; tap < 9; ++tap) w[(size_t)co * K + tap * ci_n + ci] = src[off + ((size_t)co * ci_n + ci) * 9 + tap];
      off += (size_t)co_n * ci_n * 9;
      if ((e = cudaMemcpy(which == 0 ? n->mw[l] : n->vw[l], w.data(), w.size() * 4, cudaMemcpyHostToDevice)) ||
          (e = cudaMemcpy(which == 0 ? n->mb[l] : n->vb[l], src + off, (size_t)co_n * 4, cudaMemcpyHostToDevice)))
        return cnn_fail(e, "set_adam");
      off += co_n;
    }
  }
  n->step = (int)step;
  return ILS_OK;
}

// gradients in the same order as the parameters
ils_status ils_cnn_get_grads(const ils_cnn* n, float* grads, long long count) {
  if (n == nullptr || grads == nullptr || count != (long long)param_count()) return ILS_ERR_INVALID_ARG;
  size_t off = 0;
  cudaError_t e;
  if ((e = cudaDeviceSynchronize())) return cnn_fail(e, "get_grads");
  for (int l = 0; l < kLayers; ++l) {
    const int co_n = kCout[l], ci_n = kCin[l], K = kpad(l);
    std::vector<float> w((size_t)co_n * K);
    if ((e = cudaMemcpy(w.data(), n->gw[l], w.size() * 4, cudaMemcpyDeviceToHost))) return cnn_fail(e, "get_grads");
    for (int co = 0; co < co_n; ++co)
      for (int ci = 0; ci < ci_n; ++ci)
        for (int tap = 0; tap < 9; ++tap) grads[off + ((size_t)co * ci_n + ci) * 9 + tap] = w[(size_t)co * K + tap * ci_n + ci];
    off += (size_t)co_n * ci_n * 9;
    if ((e = cudaMemcpy(grads + off, n->gb[l], (size_t)co_n * 4, cudaMemcpyDeviceToHost))) return cnn_fail(e, "get_grads");
    off += co_n;
  }
  return ILS_OK;
}

// u0 = f + net(f); f, u0: device B x 3 x H x W FP32.  Keeps the hidden activations for backward.
ils_status ils_cnn_forward(ils_cnn* n, int B, int H, int W, const float* f, float* u0, void* stream) {
  if (!cnn_shape_ok(n, B, H, W) || f == nullptr || u0 == nullptr || f == u0 || !n->packed) return ILS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const dim3 grid = tile_grid(B, H, W);
  ConvArgs a{};
  a.B = B; a.H = H; a.W = W;
  // layer 0: planar 3 -> 32, ReLU (tcgen05: f packed into 8-channel NHWC rows first)
  if (n->tc) {
    planar3_to_nhwc8(f, B, H, W, n->pkf, st, n->pk32[0]);  // pk32[0]: layer 0's weight gradient
    cudaError_t e = ils::launch_conv3_tc(B, H, W, n->pkf, n->wf[0], n->b[0], n->act[0], nullptr, 1, n->err, st);
    if (e != cudaSuccess) return cnn_fail(e, "tensor-core conv launch");
  } else {
    a.in_planar = f; a.wt = n->wf[0]; a.bias = n->b[0]; a.out_nhwc = n->act[0]; a.relu = 1; a.cout = 32;
    conv_fwd_kernel<true, 4, false><<<grid, NTHREADS, conv_smem(true, 4), st>>>(a);
  }
  for (int l = 1; l < kLayers - 1; ++l) {
    if (n->tc) {
      cudaError_t e = ils::launch_conv32_tc(B, H, W, n->act[l - 1], n->wf[l], n->b[l], n->act[l], nullptr, 1, n->err, st);
      if (e != cudaSuccess) return cnn_fail(e, "tensor-core conv launch");
      continue;
    }
    ConvArgs m{};
    m.B = B; m.H = H; m.W = W; m.in_nhwc = n->act[l - 1]; m.wt = n->wf[l]; m.bias = n->b[l];
    m.out_nhwc = n->act[l]; m.relu = 1; m.cout = 32;
    conv_fwd_kernel<false, 4, false><<<grid, NTHREADS, conv_smem(false, 4), st>>>(m);
  }
  if (n->tc) {  // layer 5: 32 -> 3 plus the residual f
    cudaError_t e = ils::launch_conv_last_tc(B, H, W, n->act[kLayers - 2], n->wf[kLayers - 1], n->b[kLayers - 1], f,
                                             u0, n->err, st);
    if (e != cudaSuccess) return cnn_fail(e, "tensor-core conv launch");
  } else {
    ConvArgs z{};
    z.B = B; z.H = H; z.W = W; z.in_nhwc = n->act[kLayers - 2]; z.wt = n->wf[kLayers - 1]; z.bias = n->b[kLayers - 1];
    z.out_planar = u0; z.resid = f; z.cout = 3;
    conv_fwd_kernel<false, 1, true><<<grid, NTHREADS, conv_smem(false, 1), st>>>(z);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ILS_OK : cnn_fail(e, "cnn forward launch");
}

// u0 = f + net(f), inference: the layer-by-layer forward, or (ILS_CNN_FUSED=1, with tcgen05)
// two fused tcgen05 kernels (layers 1-3 and 4-6, the 32-channel map between them in act[2]).
ils_status ils_cnn_infer(ils_cnn* n, int B, int H, int W, const float* f, float* u0, void* stream) {
  if (!cnn_shape_ok(n, B, H, W) || f == nullptr || u0 == nullptr || f == u0 || !n->packed) return ILS_ERR_INVALID_ARG;
  // The layer-by-layer tcgen05 kernels are the default: at 1080p RGB 402 us against 505 us for
  // the two fused kernels (bit-identical results).  ILS_CNN_FUSED=1 selects the fused kernels.
  const char* fused = getenv("ILS_CNN_FUSED");
  if (!n->tc || !(fused != nullptr && fused[0] == '1')) return ils_cnn_forward(n, B, H, W, f, u0, stream);
  const void* w[kLayers];
  const float* bias[kLayers];
  for (int l = 0; l < kLayers; ++l) {
    w[l] = n->wf[l];
    bias[l] = n->b[l];
  }
  cudaError_t e = ils::launch_warm_fused(B, H, W, f, n->act[2], u0, w, bias, n->err, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? ILS_OK : cnn_fail(e, "fused inference launch");
}

// Waits for the device and reports (then clears) a timeout raised by a tensor-core kernel.
ils_status ils_cnn_check(ils_cnn* n) {
  if (n == nullptr) return ILS_ERR_INVALID_ARG;
  int flag = 0;
  cudaError_t e = cudaMemcpy(&flag, n->err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cnn_fail(e, "ils_cnn_check");
  if (flag) {
    cudaMemset(n->err, 0, sizeof(int));
    return ILS_ERR_TIMEOUT;
  }
  return ILS_OK;
}

int ils_cnn_uses_tcgen05(const ils_cnn* n) { return n != nullptr && n->tc ? 1 : 0; }

ils_status ils_cnn_zero_grad(ils_cnn* n, void* stream) {
  if (n == nullptr) return ILS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const ParamSet ps = cnn_params(n);
  zero_all_kernel<<<(ps.start[ps.count] + 255) / 256, 256, 0, st>>>(ps);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ILS_OK : cnn_fail(e, "zero_grad");
}

// Adds dL/dparams for dL/du0 (planar FP32, B x 3 x H x W) to the gradients, using the
// activations of the last forward call on the same f.
ils_status ils_cnn_backward(ils_cnn* n, int B, int H, int W, const float* f, const float* grad_u0, void* stream) {
  if (!cnn_shape_ok(n, B, H, W) || f == nullptr || grad_u0 == nullptr || !n->packed) return ILS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const dim3 grid = tile_grid(B, H, W);
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int tiles = grid.x * grid.y * grid.z;
  const int wg_grid = tiles < 2 * sms ? tiles : 2 * sms;
  cudaError_t tc_err = cudaSuccess;
  auto wgrad = [&](int l, const bf16* dy_nhwc, const float* dy_planar) {
    WgradArgs w{};
    w.B = B; w.H = H; w.W = W; w.dy_nhwc = dy_nhwc; w.dy_planar = dy_planar;
    w.dw = n->gw[l]; w.db = n->gb[l]; w.cout = kCout[l]; w.tiles_x = grid.x; w.tiles_y = grid.y;
    if (n->tc) {
      // every layer on tcgen05; a 3-channel side (f for layer 0, dL/du0 for layer 5) is packed
      // into NHWC rows of 32 channels (channels 3-31 zero), rounded to BF16 as the mma.sync path
      // stages it; dL/du0 also into rows of 8 for layer 5's input gradient below
      cudaError_t e;
      if (l == 0) {  // f as the forward packed it (the activations are the forward's too)
        e = ils::launch_wgrad_tc(B, H, W, n->pk32[0], 32, 3, dy_nhwc, 32, 32, n->gw[l], kpad(l), n->gb[l], n->err,
                                 st);
      } else if (dy_planar != nullptr) {
        planar3_to_nhwc8(dy_planar, B, H, W, n->pk8, st, n->pk32[1]);
        e = ils::launch_wgrad_tc(B, H, W, n->act[l - 1], 32, 32, n->pk32[1], 32, kCout[l], n->gw[l], kpad(l),
                                 n->gb[l], n->err, st);
      } else {
        e = ils::launch_wgrad_tc(B, H, W, n->act[l - 1], 32, 32, dy_nhwc, 32, 32, n->gw[l], kpad(l), n->gb[l], n->err,
                                 st);
      }
      if (e != cudaSuccess && tc_err == cudaSuccess) tc_err = e;
    } else if (l == 0) {
      w.in_planar = f;
      conv_wgrad_kernel<true, false><<<wg_grid, NTHREADS, wgrad_smem(true), st>>>(w);
    } else {
      w.in_nhwc = n->act[l - 1];
      if (dy_planar != nullptr)
        conv_wgrad_kernel<false, true><<<wg_grid, NTHREADS, wgrad_smem(false), st>>>(w);
      else
        conv_wgrad_kernel<false, false><<<wg_grid, NTHREADS, wgrad_smem(false), st>>>(w);
    }
  };
  // layer 5 (32 -> 3): its output gradient is dL/du0 (the residual passes f through)
  wgrad(kLayers - 1, nullptr, grad_u0);
  if (n->tc) {
    // the weight gradient above left dL/du0 packed in pk8
    cudaError_t e = ils::launch_conv3_tc(B, H, W, n->pk8, n->wd[kLayers - 1], nullptr, n->gact[0], n->act[kLayers - 2],
                                         0, n->err, st);
    if (e != cudaSuccess) return cnn_fail(e, "tensor-core conv launch");
  } else {
    ConvArgs a{};
    a.B = B; a.H = H; a.W = W; a.in_planar = grad_u0; a.wt = n->wd[kLayers - 1];
    a.out_nhwc = n->gact[0]; a.mask = n->act[kLayers - 2]; a.cout = 32;
    conv_fwd_kernel<true, 4, false><<<grid, NTHREADS, conv_smem(true, 4), st>>>(a);
  }
  int cur = 0;
  for (int l = kLayers - 2; l >= 1; --l) {
    wgrad(l, n->gact[cur], nullptr);
    if (n->tc) {
      cudaError_t e = ils::launch_conv32_tc(B, H, W, n->gact[cur], n->wd[l], nullptr, n->gact[cur ^ 1], n->act[l - 1], 0,
                                       n->err, st);
      if (e != cudaSuccess) return cnn_fail(e, "tensor-core conv launch");
      cur ^= 1;
      continue;
    }
    ConvArgs a{};
    a.B = B; a.H = H; a.W = W; a.in_nhwc = n->gact[cur]; a.wt = n->wd[l];
    a.out_nhwc = n->gact[cur ^ 1]; a.mask = n->act[l - 1]; a.cout = 32;
    conv_fwd_kernel<false, 4, false><<<grid, NTHREADS, conv_smem(false, 4), st>>>(a);
    cur ^= 1;
  }
  wgrad(0, n->gact[cur], nullptr);
  if (tc_err != cudaSuccess) return cnn_fail(tc_err, "tensor-core weight-gradient launch");
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ILS_OK : cnn_fail(e, "cnn backward launch");
}

ils_status ils_cnn_adam_step(ils_cnn* n, float lr, float beta1, float beta2, float eps, void* stream) {
  if (n == nullptr || !(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) ||
      !(eps > 0.0f))
    return ILS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  n->step += 1;
  const float c1 = 1.0f - std::pow(beta1, (float)n->step), c2 = 1.0f - std::pow(beta2, (float)n->step);
  const ParamSet ps = cnn_params(n);
  adam_all_kernel<<<(ps.start[ps.count] + 255) / 256, 256, 0, st>>>(ps, lr, beta1, beta2, eps, c1, c2);
  cudaError_t e = cnn_pack(n, st);
  return e == cudaSuccess ? ILS_OK : cnn_fail(e, "adam step");
}

// grad = 2 (u0 - target) / n; *loss (device FP32, caller zeroes it) += mean squared error
ils_status ils_mse(const float* u0, const float* target, float* grad, long long n, float* loss, void* stream) {
  if (u0 == nullptr || target == nullptr || grad == nullptr || loss == nullptr || n < 1) return ILS_ERR_INVALID_ARG;
  mse_kernel<<<1024, 256, 0, static_cast<cudaStream_t>(stream)>>>(u0, target, grad, (size_t)n, 1.0f / (float)n, loss);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ILS_OK : cnn_fail(e, "mse");
}

}  // extern "C"
