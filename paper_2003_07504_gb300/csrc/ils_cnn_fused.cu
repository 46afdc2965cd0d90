// Warm-start network inference, u0 = f + net(f), in two fused kernels on the 5th-generation
// tensor cores: layers 1-3 (3 -> 32 -> 32 -> 32) and layers 4-6 (32 -> 32 -> 32 -> 3, plus
// the residual f).  Within a kernel the hidden activations of a tile stay in shared and
// tensor memory; only the 32-channel map between the two kernels goes through HBM (BF16
// NHWC).  Numerics are those of the layer-by-layer kernels: BF16 inputs, weights and hidden
// activations, FP32 accumulation, FP32 residual.
//
// Tile: 12 output rows x 122 output pixels.  Each layer of a kernel is computed on a region
// 128 pixels wide (the output columns and a 3-pixel margin on each side) and on the rows its
// successors need: 16, 14 and 12 rows for the three layers, one row = one MMA M-block of
// 128 pixels (GEMM view per block: M = 128 pixels, N = output channels, K = 9 taps x input
// channels).  The region is stored row-major (128 pixels per row) in the chunk-major layout
// of the other tensor-core kernel, byte (8-channel chunk c, pixel p) = c * PLANE + p * 16,
// so tap (dy, dx) of output row i is the operand that starts at pixel (i + dy - 1) * 128 +
// dx - 1: a descriptor offset.  Pixel 0 of a row then reads the previous row's last pixel
// and pixel 127 the next row's first; those wrong values creep inward one pixel per layer
// and stay inside the margin.  Pixels outside the image are zero (the convolutions' zero
// padding): written as zeros when f is staged, by TMA's out-of-bounds fill for the middle
// map, and by the epilogues for hidden activations.
//
// A layer's whole output (at most 16 blocks x 32 FP32 columns = all 512 columns of tensor
// memory) is accumulated before the epilogue drains it, so the epilogue (bias, ReLU, zero
// outside the image, BF16) can write the layer's output over its input in the one shared
// activation buffer.
//
// The 3-channel first layer pairs two taps in one K = 16 step: its input has a single
// 8-channel chunk (channels 3-7 zero), and the operand's K-direction core-matrix offset
// (LBO) points at the second tap's pixel instead of at a second channel chunk: 1 pixel for
// taps (dy, dx), (dy, dx + 1) and 126 pixels for taps (0, 2), (1, 0), so the 9 taps take 5
// MMAs (the tenth tap slot has zero weights).  The 3-channel last layer runs with N = 16
// (the smallest N of an M = 128 MMA).
//
// Every mbarrier wait is bounded; on timeout the kernel raises the error flag, waits (also
// bounded) for its own copies and MMAs in flight, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>

#include "ils_internal.h"
#include "ils_tc.cuh"

namespace ils {
namespace cnn_fused {

using namespace tc;
typedef __nv_bfloat16 bf16;

constexpr int RW = 128;                      // region width = pixels per M-block
constexpr int MARGIN = 3;                    // one pixel per fused layer
constexpr int OUT_W = RW - 2 * MARGIN;       // 122 output pixels per tile row
constexpr int OUT_H = 12;                    // output rows per tile
constexpr int IN_ROWS = OUT_H + 2 * MARGIN;  // 18 region rows of input
constexpr int GUARD = 8;                     // pixels before and after each chunk plane
constexpr int plane_bytes(int rows) { return (rows * RW + 2 * GUARD) * 16; }
constexpr int P18 = plane_bytes(IN_ROWS);       // 37120
constexpr int P16 = plane_bytes(IN_ROWS - 2);   // 33024
constexpr int WMID = 36 * 32 * 16;              // K = 288 as 36 chunks x 32 output channels
constexpr int WFIRST = 10 * 32 * 16;            // 10 tap chunks x 32 output channels
constexpr int WLAST = 36 * 16 * 16;             // 36 chunks x 16 (3 used) output channels
constexpr int NTHR = 256;
constexpr int TMA_BYTES = 4 * IN_ROWS * RW * 16;  // 147456 bytes per tile (layers 4-6)

// shared-memory layouts (byte offsets; multiples of 128)
constexpr int A_FBUF = 0, A_ACT = A_FBUF + P18, A_W0 = A_ACT + 4 * P16, A_W1 = A_W0 + WFIRST, A_W2 = A_W1 + WMID,
              A_BIAS = A_W2 + WMID, A_BAR = A_BIAS + 96 * 4, A_SMEM = A_BAR + 64;
constexpr int B_ACT = 0, B_W0 = 4 * P18, B_W1 = B_W0 + WMID, B_W2 = B_W1 + WMID, B_BIAS = B_W2 + WLAST,
              B_BAR = B_BIAS + 96 * 4, B_SMEM = B_BAR + 64;
static_assert(A_SMEM <= 227 * 1024 && B_SMEM <= 227 * 1024, "shared memory budget");
static_assert(P18 % 128 == 0 && P16 % 128 == 0 && A_W0 % 128 == 0 && B_W0 % 128 == 0, "alignment");

constexpr uint32_t kId32 = idesc_bf16(128, 32), kId16 = idesc_bf16(128, 16);  // N: multiple of 16 at M = 128

struct FusedArgs {
  int B, H, W;
  const float* f;       // B x 3 x H x W FP32 (input of layer 1, residual of layer 6)
  bf16* act;            // B x H x W x 32 BF16: layer-3 output
  float* u0;            // B x 3 x H x W FP32 output
  const bf16* w[3];     // forward GEMM rows of the kernel's three layers ([co_pad][k])
  const float* bias[3];
  int* error;           // set to 1 when a bounded wait gave up
  uint32_t spin;        // poll limit of the per-tile waits
};

// ---------------------------------------------------------------- prologue helpers

// 32-output layer, K = 288 (column k = tap * 32 + ci) -> [K chunk][co][8]
__device__ void load_w_mid(unsigned char* dst, const bf16* w) {
  for (int q = threadIdx.x; q < 36 * 32; q += blockDim.x) {
    const int kc = q >> 5, co = q & 31;
    *reinterpret_cast<uint4*>(dst + q * 16) = *reinterpret_cast<const uint4*>(w + co * 288 + kc * 8);
  }
}
// 3-output last layer (8 padded rows of 288) -> [K chunk][co < 16][8], rows 8-15 zero
__device__ void load_w_last(unsigned char* dst, const bf16* w) {
  for (int q = threadIdx.x; q < 36 * 16; q += blockDim.x) {
    const int kc = q >> 4, co = q & 15;
    *reinterpret_cast<uint4*>(dst + q * 16) =
        co < 8 ? *reinterpret_cast<const uint4*>(w + co * 288 + kc * 8) : make_uint4(0, 0, 0, 0);
  }
}
// 3-input first layer (rows of 32 columns, k = tap * 3 + ci) -> chunk q = tap q (channels
// 0-2 of the chunk; chunk 9 zero) as [chunk][co][8]
__device__ void load_w_first(unsigned char* dst, const bf16* w) {
  for (int q = threadIdx.x; q < 10 * 32; q += blockDim.x) {
    const int kc = q >> 5, co = q & 31;
    __align__(16) bf16 v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __float2bfloat16_rn(0.0f);
    if (kc < 9)
#pragma unroll
      for (int ci = 0; ci < 3; ++ci) v[ci] = w[co * 32 + kc * 3 + ci];
    *reinterpret_cast<uint4*>(dst + q * 16) = *reinterpret_cast<const uint4*>(v);
  }
}
__device__ void zero_guards(unsigned char* plane0, int nplanes, int plane, int rows) {
  const uint4 z = make_uint4(0, 0, 0, 0);
  for (int q = threadIdx.x; q < nplanes * 2 * GUARD; q += blockDim.x) {
    const int p = q / (2 * GUARD), g = q - p * 2 * GUARD;
    const int px = g < GUARD ? g : GUARD + rows * RW + (g - GUARD);
    *reinterpret_cast<uint4*>(plane0 + (size_t)p * plane + px * 16) = z;
  }
}

// ---------------------------------------------------------------- MMA issue
// Lane 0 of each of warps 0-3 issues the MMAs of the blocks m = warp (mod 4) and commits
// them to the layer's barrier (4 arrivals): one thread issues an MMA about every 50 cycles,
// about three times what a K = 16, N = 32 MMA takes on the tensor core.
constexpr int ISSUERS = 4;

// 32 -> N layer, blocks m0, m0 + 4, ... < nm; block m reads input rows in_row0 + m + dy.
__device__ __forceinline__ void issue_mid(uint32_t tmem, int m0, int nm, uint32_t act_s, int plane, int in_row0,
                                          uint32_t w_s, uint32_t idesc, int ncols, int wchunk) {
  uint64_t da[18], db[18];
#pragma unroll
  for (int tap = 0; tap < 9; ++tap) {
    const int dy = tap / 3, dx = tap % 3;
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
      const uint32_t a = act_s + kk * 2 * plane + (uint32_t)((GUARD + (in_row0 + dy) * RW + dx - 1) * 16);
      da[tap * 2 + kk] = smem_desc(a, plane, 128);
      db[tap * 2 + kk] = smem_desc(w_s + (uint32_t)((tap * 4 + kk * 2) * wchunk), wchunk, 128);
    }
  }
  for (int m = m0; m < nm; m += ISSUERS) {
#pragma unroll
    for (int s = 0; s < 18; ++s) mma_f16(tmem + m * ncols, da[s] + (uint64_t)(m * RW), db[s], idesc, s > 0 ? 1u : 0u);
  }
}

// 3 -> 32 first layer, blocks m0, m0 + 4, ... < 16 over the staged f plane (rows m + dy),
// taps paired.
__device__ __forceinline__ void issue_first(uint32_t tmem, int m0, uint32_t f_s, uint32_t w_s) {
  uint64_t da[5], db[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const int t = 2 * i, dy = t / 3, dx = t % 3;
    const int lbo_px = i == 4 ? 1 : ((t + 1) / 3 - dy) * RW + ((t + 1) % 3 - dx);
    da[i] = smem_desc(f_s + (uint32_t)((GUARD + dy * RW + dx - 1) * 16), (uint32_t)(lbo_px * 16), 128);
    db[i] = smem_desc(w_s + (uint32_t)(2 * i * 512), 512, 128);
  }
  for (int m = m0; m < IN_ROWS - 2; m += ISSUERS) {
#pragma unroll
    for (int i = 0; i < 5; ++i) mma_f16(tmem + m * 32, da[i] + (uint64_t)(m * RW), db[i], kId32, i > 0 ? 1u : 0u);
  }
}

// Warps 0-3 stay converged around their lane 0's issue; `issue(m0)` issues blocks m0 (mod 4).
template <class F>
__device__ __forceinline__ void issue_layer(uint32_t mma_bar, F&& issue) {
  const int warp = threadIdx.x >> 5;
  if (warp < ISSUERS) {
    if ((threadIdx.x & 31) == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      issue(warp);
      mma_commit(mma_bar);
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------- epilogues (all 8 warps)
// Thread -> pixel j = 32 (warp % 4) + lane of each block (its tensor-memory lane quadrant),
// channels 16 (warp / 4) .. + 15.

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// bias + ReLU (+ zero when !keep) -> 16 BF16 as two 16-byte words
__device__ __forceinline__ void pack16(const uint32_t (&r)[16], const float* bias, bool keep, uint4 (&o)[2]) {
  uint32_t* ow = reinterpret_cast<uint32_t*>(o);
#pragma unroll
  for (int c = 0; c < 16; c += 2) {
    float v0 = fmaxf(__uint_as_float(r[c]) + bias[c], 0.0f);
    float v1 = fmaxf(__uint_as_float(r[c + 1]) + bias[c + 1], 0.0f);
    if (!keep) v0 = v1 = 0.0f;
    __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
    ow[c >> 1] = *reinterpret_cast<uint32_t*>(&h);
  }
}

// Hidden layer: blocks 0..nm-1 -> chunk planes at row row0 + m; image row of block m is
// ybase + m, image column of pixel j is xbase + j.
__device__ __forceinline__ void drain_hidden(uint32_t tmem, int nm, unsigned char* act, int plane, int row0,
                                             const float* bias, int ybase, int xbase, int H, int W) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = warp & 3, h = warp >> 2, j = q * 32 + lane;
  const int X = xbase + j;
  const bool xin = X >= 0 && X < W;
  const uint32_t lane_off = (uint32_t)(q * 32) << 16;
  for (int m = 0; m < nm; m += 2) {
    uint32_t r0[16], r1[16];
    tmem_ld16(tmem + m * 32 + 16 * h + lane_off, r0);
    if (m + 1 < nm) tmem_ld16(tmem + (m + 1) * 32 + 16 * h + lane_off, r1);
    tmem_wait_ld();
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      if (m + k >= nm) break;
      const int Y = ybase + m + k;
      uint4 o[2];
      pack16(k == 0 ? r0 : r1, bias + 16 * h, xin && Y >= 0 && Y < H, o);
      unsigned char* p = act + (size_t)(GUARD + (row0 + m + k) * RW + j) * 16;
      *reinterpret_cast<uint4*>(p + (2 * h) * plane) = o[0];
      *reinterpret_cast<uint4*>(p + (2 * h + 1) * plane) = o[1];
    }
  }
}

// Layer 3 -> global NHWC BF16 for the tile's output pixels (block m = image row y0 + m).
__device__ __forceinline__ void drain_to_global(uint32_t tmem, bf16* act, const float* bias, int b, int y0, int xbase,
                                                int H, int W) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = warp & 3, h = warp >> 2, j = q * 32 + lane;
  const int X = xbase + j;
  const bool xok = j >= MARGIN && j < RW - MARGIN && X < W;
  const uint32_t lane_off = (uint32_t)(q * 32) << 16;
  for (int m = 0; m < OUT_H; m += 2) {
    uint32_t r0[16], r1[16];
    tmem_ld16(tmem + m * 32 + 16 * h + lane_off, r0);
    tmem_ld16(tmem + (m + 1) * 32 + 16 * h + lane_off, r1);
    tmem_wait_ld();
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int Y = y0 + m + k;
      if (!xok || Y >= H) continue;
      uint4 o[2];
      pack16(k == 0 ? r0 : r1, bias + 16 * h, true, o);
      uint4* dst = reinterpret_cast<uint4*>(act + (((size_t)b * H + Y) * W + X) * 32 + 16 * h);
      dst[0] = o[0];
      dst[1] = o[1];
    }
  }
}

// Layer 6 (N = 16, channels 0-2 used): u0 = f + conv + bias for the tile's output pixels;
// warps 0-3.  All of the tile's f values are loaded before the first store to u0.
__device__ __forceinline__ void drain_out(uint32_t tmem, const float* bias, const float* f, float* u0, int b, int y0,
                                          int xbase, int H, int W) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp >= 4) return;
  const int j = warp * 32 + lane;
  const int X = xbase + j;
  const bool xok = j >= MARGIN && j < RW - MARGIN && X < W;
  const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
  const size_t hw = (size_t)H * W;
  const size_t base0 = (size_t)b * 3 * hw + (size_t)y0 * W + X;
  float fv[OUT_H][3];
#pragma unroll
  for (int m = 0; m < OUT_H; ++m) {
    const bool ok = xok && y0 + m < H;
#pragma unroll
    for (int c = 0; c < 3; ++c) fv[m][c] = ok ? f[base0 + (size_t)m * W + c * hw] : 0.0f;
  }
#pragma unroll
  for (int m = 0; m < OUT_H; m += 2) {
    uint32_t r0[8], r1[8];
    tmem_ld8(tmem + m * 16 + lane_off, r0);
    tmem_ld8(tmem + (m + 1) * 16 + lane_off, r1);
    tmem_wait_ld();
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      if (!xok || y0 + m + k >= H) continue;
      const size_t base = base0 + (size_t)(m + k) * W;
#pragma unroll
      for (int c = 0; c < 3; ++c) u0[base + c * hw] = fv[m + k][c] + (__uint_as_float(k == 0 ? r0[c] : r1[c]) + bias[c]);
    }
  }
}

__device__ __forceinline__ void sync_after_epilogue() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
}

struct TileDecode {
  int b, y0, x0;
};
__device__ __forceinline__ TileDecode decode_tile(int tile, int H, int W) {
  const int tx_n = (W + OUT_W - 1) / OUT_W, ty_n = (H + OUT_H - 1) / OUT_H;
  TileDecode d;
  d.b = tile / (tx_n * ty_n);
  const int r = tile - d.b * tx_n * ty_n;
  const int ty = r / tx_n;
  d.y0 = ty * OUT_H;
  d.x0 = (r - ty * tx_n) * OUT_W;
  return d;
}

// Shared prologue: tensor memory (all 512 columns) and the MMA barrier.
__device__ __forceinline__ uint32_t setup_tmem(uint32_t* slot) {
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(saddr(slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  return *slot;
}
__device__ __forceinline__ void teardown(uint32_t tmem, int* s_abort, int* error) {
  if (threadIdx.x == 0 && *s_abort) atomicExch(error, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
}

// Outstanding-work bookkeeping of a CTA: the parity of the next phase of a barrier and
// whether a phase that was started (commit or copy issued) has not been observed yet.
struct Phase {
  uint32_t next = 0, open_par = 0;
  bool open = false;
  __device__ __forceinline__ void started() {
    open = true;
    open_par = next;
  }
  // bounded wait for the started phase; a timeout marks the CTA aborted and leaves it open
  __device__ __forceinline__ void wait(uint32_t bar, uint32_t spin, int* s_abort) {
    if (mbar_wait(bar, next, spin)) open = false;
    else *s_abort = 1;
    next ^= 1;
  }
  // before tensor memory is freed or the CTA exits: observe an open phase (bounded)
  __device__ __forceinline__ void drain(uint32_t bar) {
    if (open) mbar_wait(bar, open_par);
  }
};

// all threads wait for the MMA phase, then order their tensor-memory reads after it
__device__ __forceinline__ void wait_mma(uint32_t bar, Phase& ph, uint32_t spin, int* s_abort) {
  ph.wait(bar, spin, s_abort);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// ---------------------------------------------------------------- layers 1-3

// f (BF16, channels 0-2 of one 8-channel chunk; zero outside the image) of a tile's region
__device__ __forceinline__ void stage_f(const FusedArgs& a, const TileDecode& t, unsigned char* fbuf) {
  const size_t hw = (size_t)a.H * a.W;
  const int xb = t.x0 - MARGIN, yb = t.y0 - MARGIN;
  for (int idx = threadIdx.x; idx < IN_ROWS * RW; idx += NTHR) {
    const int Y = yb + (idx >> 7), X = xb + (idx & (RW - 1));
    float v[3] = {0.0f, 0.0f, 0.0f};
    if (Y >= 0 && Y < a.H && X >= 0 && X < a.W) {
      const float* p = a.f + (size_t)t.b * 3 * hw + (size_t)Y * a.W + X;
      v[0] = p[0];
      v[1] = p[hw];
      v[2] = p[2 * hw];
    }
    __align__(16) __nv_bfloat162 h[4];
    h[0] = __floats2bfloat162_rn(v[0], v[1]);
    h[1] = __floats2bfloat162_rn(v[2], 0.0f);
    h[2] = h[3] = __floats2bfloat162_rn(0.0f, 0.0f);
    *reinterpret_cast<uint4*>(fbuf + (size_t)(GUARD + idx) * 16) = *reinterpret_cast<const uint4*>(h);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__global__ void __launch_bounds__(NTHR, 1) warm_l123_kernel(FusedArgs a) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  unsigned char* fbuf = sm + A_FBUF;
  unsigned char* act = sm + A_ACT;
  float* bias = reinterpret_cast<float*>(sm + A_BIAS);
  const uint32_t mma_bar = saddr(sm + A_BAR);
  const uint32_t f_s = saddr(fbuf), act_s = saddr(act);
  const int tid = threadIdx.x;

  load_w_first(sm + A_W0, a.w[0]);
  load_w_mid(sm + A_W1, a.w[1]);
  load_w_mid(sm + A_W2, a.w[2]);
  for (int i = tid; i < 96; i += NTHR) bias[i] = a.bias[i >> 5][i & 31];
  zero_guards(fbuf, 1, P18, IN_ROWS);
  zero_guards(act, 4, P16, IN_ROWS - 2);
  if (tid == 0) {
    mbar_init(mma_bar, ISSUERS);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const int ntiles = a.B * ((a.W + OUT_W - 1) / OUT_W) * ((a.H + OUT_H - 1) / OUT_H);
  if ((int)blockIdx.x < ntiles) stage_f(a, decode_tile(blockIdx.x, a.H, a.W), fbuf);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  const uint32_t tmem = setup_tmem(&s_tmem);

  Phase mph;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const TileDecode t = decode_tile(tile, a.H, a.W);
    const int xb = t.x0 - MARGIN, yb = t.y0 - MARGIN;  // image position of region pixel (0, 0)
    // layer 1: region rows 1..16 -> activation rows 0..15
    issue_layer(mma_bar, [&](int m0) { issue_first(tmem, m0, f_s, saddr(sm + A_W0)); });
    mph.started();
    wait_mma(mma_bar, mph, a.spin, &s_abort);
    drain_hidden(tmem, IN_ROWS - 2, act, P16, 0, bias, yb + 1, xb, a.H, a.W);
    sync_after_epilogue();
    if (s_abort) break;
    // layer 2: region rows 2..15 (activation rows 1..14), reads activation rows m .. m+2;
    // meanwhile the next tile's f is staged (layer 1, its only reader, is done)
    issue_layer(mma_bar, [&](int m0) {
      issue_mid(tmem, m0, IN_ROWS - 4, act_s, P16, 0, saddr(sm + A_W1), kId32, 32, 512);
    });
    mph.started();
    if (tile + (int)gridDim.x < ntiles) stage_f(a, decode_tile(tile + gridDim.x, a.H, a.W), fbuf);
    wait_mma(mma_bar, mph, a.spin, &s_abort);
    drain_hidden(tmem, IN_ROWS - 4, act, P16, 1, bias + 32, yb + 2, xb, a.H, a.W);
    sync_after_epilogue();
    if (s_abort) break;
    // layer 3: region rows 3..14 = the output rows, reads activation rows m+1 .. m+3
    issue_layer(mma_bar, [&](int m0) {
      issue_mid(tmem, m0, OUT_H, act_s, P16, 1, saddr(sm + A_W2), kId32, 32, 512);
    });
    mph.started();
    wait_mma(mma_bar, mph, a.spin, &s_abort);
    drain_to_global(tmem, a.act, bias + 64, t.b, t.y0, xb, a.H, a.W);
    sync_after_epilogue();
    if (s_abort) break;
  }
  // after a timeout: the last commits must be observed before tensor memory is freed (bounded)
  if (tid == 0) mph.drain(mma_bar);
  teardown(tmem, &s_abort, a.error);
}

// ---------------------------------------------------------------- layers 4-6

__global__ void __launch_bounds__(NTHR, 1) warm_l456_kernel(const __grid_constant__ CUtensorMap act_map, FusedArgs a) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  unsigned char* act = sm + B_ACT;
  float* bias = reinterpret_cast<float*>(sm + B_BIAS);
  const uint32_t mma_bar = saddr(sm + B_BAR), tma_bar = saddr(sm + B_BAR + 8);
  const uint32_t act_s = saddr(act);
  const int tid = threadIdx.x;

  load_w_mid(sm + B_W0, a.w[0]);
  load_w_mid(sm + B_W1, a.w[1]);
  load_w_last(sm + B_W2, a.w[2]);
  for (int i = tid; i < 96; i += NTHR) bias[i] = (i < 64 || (i & 31) < 3) ? a.bias[i >> 5][i & 31] : 0.0f;
  zero_guards(act, 4, P18, IN_ROWS);
  if (tid == 0) {
    mbar_init(mma_bar, ISSUERS);
    mbar_init(tma_bar, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  const uint32_t tmem = setup_tmem(&s_tmem);

  // the 18 x 128 region of the layer-3 map as four 8-channel chunk planes (zero fill outside)
  auto load_region = [&](int tile) {
    const TileDecode t = decode_tile(tile, a.H, a.W);
    mbar_expect_tx(tma_bar, TMA_BYTES);
    for (int c = 0; c < 4; ++c)
      tma_load_4d(act_s + c * P18 + GUARD * 16, &act_map, c * 8, t.x0 - MARGIN, t.y0 - MARGIN, t.b, tma_bar);
  };
  const int ntiles = a.B * ((a.W + OUT_W - 1) / OUT_W) * ((a.H + OUT_H - 1) / OUT_H);
  Phase mph, tph;
  if ((int)blockIdx.x < ntiles) {
    if (tid == 0) load_region(blockIdx.x);
    tph.started();
  }
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const TileDecode t = decode_tile(tile, a.H, a.W);
    const int xb = t.x0 - MARGIN, yb = t.y0 - MARGIN;
    tph.wait(tma_bar, a.spin, &s_abort);
    __syncthreads();
    if (s_abort) break;
    // layer 4: region rows 1..16 in place, reads rows m .. m+2
    issue_layer(mma_bar, [&](int m0) {
      issue_mid(tmem, m0, IN_ROWS - 2, act_s, P18, 0, saddr(sm + B_W0), kId32, 32, 512);
    });
    mph.started();
    wait_mma(mma_bar, mph, a.spin, &s_abort);
    drain_hidden(tmem, IN_ROWS - 2, act, P18, 1, bias, yb + 1, xb, a.H, a.W);
    sync_after_epilogue();
    if (s_abort) break;
    // layer 5: region rows 2..15 in place, reads rows m+1 .. m+3
    issue_layer(mma_bar, [&](int m0) {
      issue_mid(tmem, m0, IN_ROWS - 4, act_s, P18, 1, saddr(sm + B_W1), kId32, 32, 512);
    });
    mph.started();
    wait_mma(mma_bar, mph, a.spin, &s_abort);
    drain_hidden(tmem, IN_ROWS - 4, act, P18, 2, bias + 32, yb + 2, xb, a.H, a.W);
    sync_after_epilogue();
    if (s_abort) break;
    // layer 6: output rows (region rows 3..14), reads rows m+2 .. m+4, N = 16; once its
    // MMAs are done the buffer is free and the next tile's region is requested
    issue_layer(mma_bar, [&](int m0) {
      issue_mid(tmem, m0, OUT_H, act_s, P18, 2, saddr(sm + B_W2), kId16, 16, 256);
    });
    mph.started();
    wait_mma(mma_bar, mph, a.spin, &s_abort);
    __syncthreads();  // every thread has seen the layer-6 MMAs finish (or the abort)
    if (!s_abort && tile + (int)gridDim.x < ntiles) {
      if (tid == 0) load_region(tile + gridDim.x);
      tph.started();
    }
    drain_out(tmem, bias + 64, a.f, a.u0, t.b, t.y0, xb, a.H, a.W);
    sync_after_epilogue();
    if (s_abort) break;
  }
  if (tid == 0) {
    mph.drain(mma_bar);
    tph.drain(tma_bar);
  }
  teardown(tmem, &s_abort, a.error);
}

}  // namespace cnn_fused

// ---------------------------------------------------------------- host side

cudaError_t warm_fused_set_attributes() {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(cnn_fused::warm_l123_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                cnn_fused::A_SMEM)))
    return e;
  return cudaFuncSetAttribute(cnn_fused::warm_l456_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              cnn_fused::B_SMEM);
}

// u0 = f + net(f) for B x 3 x H x W FP32 images; act: a B x H x W x 32 BF16 scratch map.
// w[l], bias[l]: the six layers' forward GEMM rows and biases.
cudaError_t launch_warm_fused(int B, int H, int W, const float* f, void* act, float* u0, const void* const* w,
                              const float* const* bias, int* error, cudaStream_t st) {
  using namespace cnn_fused;
  CUtensorMap map;
  if (!make_nhwc32_map(&map, act, B, H, W, RW, IN_ROWS)) return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long tiles = (long long)B * ((W + OUT_W - 1) / OUT_W) * ((H + OUT_H - 1) / OUT_H);
  const int grid = (int)(tiles < sms ? tiles : sms);  // persistent: one CTA per SM
  const char* spin = getenv("ILS_TEST_TC_SPIN");      // test hook: tiny poll limit -> timeout path
  FusedArgs a{};
  a.B = B; a.H = H; a.W = W;
  a.f = f;
  a.act = static_cast<bf16*>(act);
  a.u0 = u0;
  a.error = error;
  a.spin = (spin != nullptr && spin[0] != 0) ? (uint32_t)atoi(spin) : kSpinLimit;
  for (int l = 0; l < 3; ++l) {
    a.w[l] = static_cast<const bf16*>(w[l]);
    a.bias[l] = bias[l];
  }
  warm_l123_kernel<<<grid, NTHR, A_SMEM, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  for (int l = 0; l < 3; ++l) {
    a.w[l] = static_cast<const bf16*>(w[3 + l]);
    a.bias[l] = bias[3 + l];
  }
  warm_l456_kernel<<<grid, NTHR, B_SMEM, st>>>(map, a);
  return cudaGetLastError();
}

}  // namespace ils
