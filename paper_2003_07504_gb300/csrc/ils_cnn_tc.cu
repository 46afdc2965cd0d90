// 3x3 convolutions of the warm-start network on the 5th-generation tensor cores (TMA -> shared
// memory -> tcgen05.mma, accumulator in tensor memory -> tcgen05.ld epilogue): the 32 -> 32
// layers and their input gradients (conv32_ring_tc_kernel), the 3 -> 32 layer and the input
// gradient of the 32 -> 3 layer (conv3_tc_kernel), and the weight gradients of every layer
// (conv32_wgrad_tc_kernel).
//
// GEMM view of a convolution tile: M = 128 consecutive output pixels of one image row, N = 32
// output channels, K = 9 taps x input channels in MMAs of K = 16 (BF16 in, FP32 accumulate).
// With 32 input channels a row of pixels x0-1 .. x0+128 is one TMA copy of 130 pixels x 64
// bytes (all 32 channels of a pixel in one 64-byte row) with the 64-byte swizzle into a
// 1024-byte-aligned row buffer.  That is the canonical 64-byte-swizzled K-major operand
// (8-pixel groups 512 bytes apart): tap (dy, dx) starts at pixel dx of the buffer of row
// y - 1 + dy and the second K half 32 bytes further.  The hardware applies the swizzle to the
// absolute shared-memory address on both sides (TMA write, MMA read), so a start inside the
// 512-byte pattern needs no base offset in the descriptor (measured: the offset
// (start >> 7) & 7 gives wrong results, 0 gives the mma.sync kernels' results).  Four copies of
// 16-byte channel chunks into a chunk-major layout (the no-swizzle form) moved the same bytes
// as 1,560 16-byte rows per tile with twice the sectors: 67 us per launch on the 16 x 256 x 256
// training batch that way, 38 us with the swizzled rows, 36 us with the row ring.  Out-of-image
// pixels come from TMA's zero fill (the convolution's zero padding).  The weights,
// [K-chunk][output channel][8] (no swizzle), stay in shared memory for all tiles of a
// persistent CTA.  A 3-channel input keeps the chunk-major form (one 8-channel plane, 16 bytes
// per pixel, rows 136 pixels apart), each image row loaded as copies of 64 and 66 pixels of
// 8-byte elements (1-KB rows instead of 130 rows of 16 bytes).
//
// The convolution kernels are persistent pipelines: one warp issues the TMA copies, one the
// MMAs into two tensor-memory accumulators, eight drain them (two per tensor-memory lane
// quarter, 16 output channels each).  Every wait on an mbarrier is bounded; on timeout the
// kernel raises a flag, waits (also bounded) for its own copies and MMAs in flight, frees its
// tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>

#include "ils_internal.h"
#include "ils_tc.cuh"

namespace ils {
namespace cnn_tc {

typedef __nv_bfloat16 bf16;

constexpr int TILE = 128;                  // pixels per tile (M)
constexpr int HALO_W = TILE + 2;           // 130
constexpr int B_CHUNKS = 36;               // K = 288 = 36 chunks of 8
constexpr int B_BYTES = B_CHUNKS * 32 * 16;  // 18432
using tc::kSpinLimit;
using tc::mbar_arrive;
using tc::mbar_expect_tx;
using tc::mbar_init;
using tc::mbar_wait;
using tc::saddr;
using tc::smem_desc;
using tc::smem_desc_sw64;
using tc::tma_load_4d;

constexpr uint32_t kIdesc = tc::idesc_bf16(128, 32);

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t accumulate) {
  tc::mma_f16(tmem_d, da, db, kIdesc, accumulate);
}
using tc::mma_commit;

struct TcArgs {
  int B, H, W;
  const bf16* wt;     // [32 co][288] BF16, column k = tap * 32 + ci (as for the mma.sync kernels);
                      // IN8: [32 co][32], column k = tap * 3 + ci (k < 27)
  const float* bias;  // [32] or null
  bf16* out;          // NHWC BF16
  const bf16* mask;   // NHWC BF16, or null: output zeroed where mask <= 0
  float* out_planar;  // LAST (32 -> 3): B x 3 x H x W FP32 output, out_planar = resid + conv + bias
  const float* resid;
  int relu;
  int* error;         // set to 1 when a bounded wait gave up
  uint32_t spin;      // poll limit of the per-tile waits (a test sets it tiny to exercise the timeout path)
};

// 32-channel input: a row of pixels x0-1 .. x0+128 as one TMA copy of 130 pixels x 64 bytes
// with the 64-byte swizzle, in a 1024-byte-aligned buffer
constexpr int RB = 9216;                                // bytes per row buffer (130 x 64 = 8320 used)
constexpr int NTHR = 320;                               // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue

// The 3-channel variant (IN8): the input is an NHWC row of 8 channels (3 values, 5 zeros), one
// chunk plane per stage.  A tap is then half a K = 16 step, so step j pairs taps 2j and 2j + 1:
// the descriptor starts at the first tap's pixel and its K-direction stride (LBO) is the byte
// distance to the second tap's pixel.  The ninth tap pairs with tap 7 under zero weights, so
// every operand byte read is a copied pixel.  Weights: 10 K-chunks [chunk][co][8], chunk 2j + h
// holding tap 2j + h (chunk 8 zero, chunk 9 tap 8), channels 3-7 zero.
constexpr int IN8_RPX = 136;                               // row stride in pixels (2176 bytes, 128-aligned)
constexpr int IN8_C0 = 64, IN8_C1 = HALO_W - IN8_C0;       // pixels of a row's two copies (64, 66)
constexpr int IN8_STEPS = 5;
constexpr int IN8_CHUNKS = 2 * IN8_STEPS;
constexpr int IN8_A_BYTES = 3 * IN8_RPX * 16;              // 6528
constexpr int IN8_TMA_BYTES = 3 * HALO_W * 16;             // 6240
constexpr int IN8_B_BYTES = IN8_CHUNKS * 32 * 16;          // 5120
constexpr int IN8_STAGES = 6;
constexpr int SMEM_PIPE_IN8 = 1024 + IN8_STAGES * IN8_A_BYTES + IN8_B_BYTES + 128 + 128;

__host__ __device__ constexpr int in8_tap(int chunk) { return chunk < 8 ? chunk : (chunk == 8 ? -1 : 8); }

// The 3-channel convolution (IN8 input): a persistent, warp-specialized pipeline.  Tile i
// (output row y, pixels x0 .. x0 + 127; tiles strided over the CTAs) uses input stage
// i % IN8_STAGES and accumulator i % 2 (32 tensor-memory columns each).  Barriers (phase parity from the
// use count): full[s] TMA -> MMA, empty[s] MMA -> TMA (tcgen05.commit), accf[b] MMA ->
// epilogue, acce[b] epilogue -> MMA (128 arrivals).
__global__ void __launch_bounds__(NTHR, 1) conv3_tc_kernel(const __grid_constant__ CUtensorMap in_map,
                                                           const __grid_constant__ CUtensorMap in_map2, TcArgs a) {
  constexpr int NST = IN8_STAGES;
  constexpr int ABYTES = IN8_A_BYTES;
  constexpr int BBYTES = IN8_B_BYTES;
  extern __shared__ __align__(128) unsigned char smraw[];
  // stages on a 1024-byte boundary: the 64-byte swizzle pattern repeats every 512 bytes
  unsigned char* sm = smraw + ((1024u - (saddr(smraw) & 1023u)) & 1023u);
  unsigned char* sB = sm + NST * ABYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + NST * ABYTES + BBYTES);
  float* sbias = reinterpret_cast<float*>(sm + NST * ABYTES + BBYTES + 128);
  __shared__ uint32_t tmem_base_slot;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto full = [&](int s) { return saddr(&bars[s]); };
  auto empty = [&](int s) { return saddr(&bars[NST + s]); };
  auto accf = [&](int b) { return saddr(&bars[2 * NST + b]); };
  auto acce = [&](int b) { return saddr(&bars[2 * NST + 2 + b]); };

  for (int q = threadIdx.x; q < IN8_CHUNKS * 32; q += blockDim.x) {
    const int kc = q >> 5, co = q & 31, tap = in8_tap(kc);
    uint32_t w[4] = {0u, 0u, 0u, 0u};
    if (tap >= 0) {
      const bf16* src = a.wt + co * 32 + tap * 3;
      __nv_bfloat162 c01, c2z;
      c01.x = src[0];
      c01.y = src[1];
      c2z.x = src[2];
      c2z.y = __float2bfloat16_rn(0.0f);
      w[0] = *reinterpret_cast<uint32_t*>(&c01);
      w[1] = *reinterpret_cast<uint32_t*>(&c2z);
    }
    *reinterpret_cast<uint4*>(sB + (size_t)q * 16) = make_uint4(w[0], w[1], w[2], w[3]);
  }
  if (threadIdx.x < 32) sbias[threadIdx.x] = a.bias != nullptr ? a.bias[threadIdx.x] : 0.0f;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf(b), 1);
      mbar_init(acce(b), 256);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(saddr(&tmem_base_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_slot;

  const int tiles_x = (a.W + TILE - 1) / TILE;
  const int ntiles = a.B * a.H * tiles_x;
  const int my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  bool failed = false;

  if (warp == 0 && lane == 0) {
    // ---------------- producer
    int issued = 0;
    for (int i = 0; i < my_tiles; ++i) {
      const int tile = blockIdx.x + i * gridDim.x;
      const int b = tile / (a.H * tiles_x);
      const int rr = tile - b * a.H * tiles_x;
      const int y = rr / tiles_x, x0 = (rr - y * tiles_x) * TILE;
      const int s = i % NST;
      if (i >= NST && !mbar_wait(empty(s), ((i / NST) & 1) ^ 1, a.spin)) { failed = true; break; }
      mbar_expect_tx(full(s), IN8_TMA_BYTES);
      // per row a copy of 64 and one of 66 pixels (x in 8-byte units: always even)
      for (int r = 0; r < 3; ++r) {
        const uint32_t row = saddr(sm + s * ABYTES + r * IN8_RPX * 16);
        tc::tma_load_3d(row, &in_map, 2 * (x0 - 1), y - 1 + r, b, full(s));
        tc::tma_load_3d(row + IN8_C0 * 16, &in_map2, 2 * (x0 - 1 + IN8_C0), y - 1 + r, b, full(s));
      }
      issued = i + 1;
    }
    // before the CTA may end, every copy issued must have landed (bounded)
    for (int i = (issued > NST ? issued - NST : 0); i < issued; ++i)
      if (!mbar_wait(full(i % NST), (i / NST) & 1)) failed = true;
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    // The weights' descriptors are the same for every tile, and a tile's A descriptors differ
    // from its first one only in the start-address field (address >> 4, 14 bits; every address
    // here is below 256 KB, so adding a tap's offset >> 4 never carries out of the field): one
    // 64-bit add per MMA instead of a descriptor build.
    const uint32_t b0 = saddr(sB);
    uint64_t db[IN8_STEPS];
#pragma unroll
    for (int q = 0; q < IN8_STEPS; ++q) db[q] = smem_desc(b0 + (uint32_t)(2 * q * 512), 512, 128);
    int issued = 0, s = 0, sphase = 0;  // stage of tile i and the parity of its full barrier
    for (int i = 0; i < my_tiles; ++i) {
      const int acc = i & 1;
      if (!mbar_wait(full(s), sphase, a.spin)) { failed = true; break; }
      if (i >= 2 && !mbar_wait(acce(acc), ((i >> 1) & 1) ^ 1, a.spin)) { failed = true; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = saddr(sm + s * ABYTES), d = tmem + acc * 32;
      const uint64_t da0 = smem_desc(a0, 16, 128);
#pragma unroll
      for (int j = 0; j < IN8_STEPS; ++j) {
        // taps t0 (K half 0) and t1 (K half 1) of this step; byte offset of tap t's pixel 0
        const int t0 = j < 4 ? 2 * j : 7, t1 = j < 4 ? 2 * j + 1 : 8;
        const int o0 = ((t0 / 3) * IN8_RPX + t0 % 3) * 16, o1 = ((t1 / 3) * IN8_RPX + t1 % 3) * 16;
        // the K stride (LBO, bits 16-29) is the distance between the two taps
        const uint64_t da = (da0 & ~(0x3FFFull << 16)) + (uint64_t)(o0 >> 4) + ((uint64_t)((o1 - o0) >> 4) << 16);
        mma_f16(d, da, db[j], j ? 1u : 0u);
      }
      mma_commit(empty(s));
      mma_commit(accf(acc));
      issued = i + 1;
      if (++s == NST) {
        s = 0;
        sphase ^= 1;
      }
    }
    // the MMAs issued must complete before tensor memory is freed (bounded)
    for (int i = (issued > 2 ? issued - 2 : 0); i < issued; ++i)
      if (!mbar_wait(accf(i & 1), (i >> 1) & 1)) failed = true;
  } else if (warp >= 2) {
    // ---------------- epilogue: thread -> pixel (tensor-memory lane) 32 * (warp % 4) + lane and
    // output channels 16 h .. 16 h + 15 (warps 2-5: h = 0, warps 6-9: h = 1)
    const int q = warp & 3, h16 = (warp - 2) >> 2;
    const int px = q * 32 + lane;
    for (int i = 0; i < my_tiles; ++i) {
      const int acc = i & 1;
      if (!mbar_wait(accf(acc), (i >> 1) & 1, a.spin)) { failed = true; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      uint32_t r[16];
      const uint32_t taddr = tmem + acc * 32 + h16 * 16 + ((uint32_t)(q * 32) << 16);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(acce(acc));
      const int tile = blockIdx.x + i * gridDim.x;
      const int b = tile / (a.H * tiles_x);
      const int rr = tile - b * a.H * tiles_x;
      const int y = rr / tiles_x, x = (rr - y * tiles_x) * TILE + px;
      if (x < a.W) {
        const size_t pix = ((size_t)b * a.H + y) * a.W + x;
        uint4 mk[2];
        if (a.mask != nullptr)
#pragma unroll
          for (int t = 0; t < 2; ++t) mk[t] = reinterpret_cast<const uint4*>(a.mask + pix * 32 + h16 * 16)[t];
        uint4 o[2];
        uint32_t* ow = reinterpret_cast<uint32_t*>(o);
#pragma unroll
        for (int c = 0; c < 16; c += 2) {
          const int ch = h16 * 16 + c;
          float v0 = __uint_as_float(r[c]) + sbias[ch], v1 = __uint_as_float(r[c + 1]) + sbias[ch + 1];
          if (a.relu) {
            v0 = fmaxf(v0, 0.0f);
            v1 = fmaxf(v1, 0.0f);
          }
          if (a.mask != nullptr) {
            const __nv_bfloat162 m = reinterpret_cast<const __nv_bfloat162*>(mk)[c >> 1];
            if (!(__bfloat162float(m.x) > 0.0f)) v0 = 0.0f;
            if (!(__bfloat162float(m.y) > 0.0f)) v1 = 0.0f;
          }
          __nv_bfloat162 hv = __floats2bfloat162_rn(v0, v1);
          ow[c >> 1] = *reinterpret_cast<uint32_t*>(&hv);
        }
#pragma unroll
        for (int t = 0; t < 2; ++t) reinterpret_cast<uint4*>(a.out + pix * 32 + h16 * 16)[t] = o[t];
      }
    }
  }
  if (failed) atomicExch(a.error, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem));
}

// ---------------------------------------------------------------- 32-channel input, row ring
// The same convolution with each CTA walking a contiguous range of tiles down its columns
// (tile g: column g / H, output row g % H), so that consecutive tiles share input rows: a ring
// of CR_RING row buffers (row r in buffer r mod CR_RING, 130 pixels x 64 bytes with the 64-byte
// swizzle) holds rows y - 1 .. y + 1 of the tiles in flight, and a tile needs one new row (three
// at the start of a column run).  Tap (dy, dx) of output row y is the operand at pixel dx of the
// buffer of row y - 1 + dy.  One thread issues the copies: tile g takes barrier slot j =
// (g - t0) mod CR_NT once the MMAs of the slot's previous tile (g - CR_NT) are done, which also
// were the last to read the ring buffer its new row takes (CR_RING = CR_NT + 2); a column run
// starts after every MMA issued is done.  One thread issues the MMAs into two accumulators,
// eight warps drain them as in conv3_tc_kernel.
constexpr int CR_NT = 4;
constexpr int CR_RING = CR_NT + 2;
constexpr int CR_ROWS_BYTES = CR_RING * RB;                               // 55296
constexpr int SMEM_RING = 1024 + CR_ROWS_BYTES + B_BYTES + 128 + 128;

__device__ __forceinline__ int cr_ring(int r) { return ((r % CR_RING) + CR_RING) % CR_RING; }

// LAST: the 32 -> 3 last layer with the residual, N = 16 (output channels 3-15 zero weights) and
// a planar FP32 epilogue; weights [8 padded rows][288] as the forward GEMM rows of that layer.
template <bool LAST>
__global__ void __launch_bounds__(NTHR, 1) conv32_ring_tc_kernel(const __grid_constant__ CUtensorMap in_map, TcArgs a) {
  extern __shared__ __align__(128) unsigned char smraw[];
  unsigned char* rows = smraw + ((1024u - (saddr(smraw) & 1023u)) & 1023u);  // 1024-byte aligned
  unsigned char* sB = rows + CR_ROWS_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + B_BYTES);
  float* sbias = reinterpret_cast<float*>(sB + B_BYTES + 128);
  __shared__ uint32_t tmem_base_slot;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto full = [&](int j) { return saddr(&bars[j]); };
  auto empty = [&](int j) { return saddr(&bars[CR_NT + j]); };
  auto accf = [&](int b) { return saddr(&bars[2 * CR_NT + b]); };
  auto acce = [&](int b) { return saddr(&bars[2 * CR_NT + 2 + b]); };
  auto next_slot = [](int j) { return j + 1 == CR_NT ? 0 : j + 1; };

  constexpr int NCO = LAST ? 16 : 32;  // N of the MMAs: rows of the weight chunks
  for (int q = threadIdx.x; q < B_CHUNKS * NCO; q += blockDim.x) {
    const int kc = q / NCO, co = q % NCO;
    *reinterpret_cast<uint4*>(sB + (size_t)q * 16) =
        (!LAST || co < 8) ? reinterpret_cast<const uint4*>(a.wt)[co * B_CHUNKS + kc] : make_uint4(0u, 0u, 0u, 0u);
  }
  if (threadIdx.x < 32) sbias[threadIdx.x] = a.bias != nullptr && (!LAST || threadIdx.x < 3) ? a.bias[threadIdx.x] : 0.0f;
  if (threadIdx.x == 0) {
    for (int j = 0; j < CR_NT; ++j) {
      mbar_init(full(j), 1);
      mbar_init(empty(j), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf(b), 1);
      mbar_init(acce(b), 256);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(saddr(&tmem_base_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_slot;

  const int tiles_x = (a.W + TILE - 1) / TILE;
  const int total = a.B * tiles_x * a.H;
  const int t0 = (int)((long long)total * blockIdx.x / gridDim.x);
  const int t1 = (int)((long long)total * (blockIdx.x + 1) / gridDim.x);
  // a tile's position (column col of image b at pixel x0, output row y), advanced one tile at a
  // time: a division only when a column ends
  struct Pos {
    int col, y, b, x0;
  };
  auto set_col = [&](Pos& p) {
    p.b = p.col / tiles_x;
    p.x0 = (p.col - p.b * tiles_x) * TILE;
  };
  auto start = [&](int g) {
    Pos p;
    p.col = g / a.H;
    p.y = g - p.col * a.H;
    set_col(p);
    return p;
  };
  auto advance = [&](Pos& p) {
    if (++p.y == a.H) {
      p.y = 0;
      ++p.col;
      set_col(p);
    }
  };
  bool failed = false;

  if (warp == 0 && lane == 0 && t1 > t0) {
    // ---------------- copy thread.  Per slot (bit j): loads so far mod 2, a load whose MMAs
    // this thread has not waited for, a slot loaded at least once.
    uint32_t loadpar = 0, outstanding = 0, used = 0;
    Pos ld = start(t0);
    int lj = 0;
    for (int g = t0; g < t1 && !failed; ++g) {
      const bool first = g == t0 || ld.y == 0;
      const uint32_t need = first ? outstanding : (outstanding & (1u << lj));
      for (int j = 0; j < CR_NT; ++j)
        if ((need >> j) & 1u) {
          if (!mbar_wait(empty(j), ((loadpar >> j) & 1u) ^ 1u, a.spin)) {
            failed = true;
            break;
          }
          outstanding &= ~(1u << j);
        }
      if (failed) break;
      mbar_expect_tx(full(lj), (first ? 3 : 1) * HALO_W * 64);
      for (int r = first ? ld.y - 1 : ld.y + 1; r <= ld.y + 1; ++r)
        tma_load_4d(saddr(rows + cr_ring(r) * RB), &in_map, 0, ld.x0 - 1, r, ld.b, full(lj));
      loadpar ^= 1u << lj;
      outstanding |= 1u << lj;
      used |= 1u << lj;
      advance(ld);
      lj = next_slot(lj);
    }
    // every copy issued must have landed before the CTA may end (bounded)
    for (int j = 0; j < CR_NT; ++j)
      if (((used >> j) & 1u) && !mbar_wait(full(j), ((loadpar >> j) & 1u) ^ 1u)) failed = true;
  } else if (warp == 1 && lane == 0 && t1 > t0) {
    // ---------------- MMA thread
    const uint32_t b0 = saddr(sB), rows0 = saddr(rows);
    uint64_t db[18];
#pragma unroll
    for (int q = 0; q < 18; ++q)
      db[q] = smem_desc(b0 + (uint32_t)(((q >> 1) * 4 + (q & 1) * 2) * NCO * 16), NCO * 16, 128);
    constexpr uint32_t idesc = tc::idesc_bf16(128, NCO);
    uint32_t fullpar = 0;
    Pos cur = start(t0);
    int j = 0, issued = 0;
    for (int i = 0; i < t1 - t0; ++i) {
      const int acc = i & 1;
      if (!mbar_wait(full(j), (fullpar >> j) & 1u, a.spin)) { failed = true; break; }
      fullpar ^= 1u << j;
      if (i >= 2 && !mbar_wait(acce(acc), ((i >> 1) & 1) ^ 1, a.spin)) { failed = true; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t d = tmem + acc * 32;
#pragma unroll
      for (int dy = 0; dy < 3; ++dy) {
        const uint64_t da0 = smem_desc_sw64(rows0 + (uint32_t)(cr_ring(cur.y - 1 + dy) * RB), 16, 512);
#pragma unroll
        for (int q = 0; q < 6; ++q) {  // (dx, channel half) of tap (dy, dx)
          const int dx = q >> 1, kk = q & 1;
          tc::mma_f16(d, da0 + (uint64_t)((dx * 64 + kk * 32) >> 4), db[dy * 6 + q], idesc, (dy | q) ? 1u : 0u);
        }
      }
      mma_commit(empty(j));
      mma_commit(accf(acc));
      issued = i + 1;
      advance(cur);
      j = next_slot(j);
    }
    // the MMAs issued must complete before tensor memory is freed (bounded)
    for (int i = (issued > 2 ? issued - 2 : 0); i < issued; ++i)
      if (!mbar_wait(accf(i & 1), (i >> 1) & 1)) failed = true;
  } else if (warp >= 2 && t1 > t0) {
    // ---------------- epilogue: thread -> pixel 32 * (warp % 4) + lane, channels 16 h .. + 15
    const int q = warp & 3, h16 = (warp - 2) >> 2;
    const int px = q * 32 + lane;
    Pos cur = start(t0);
    for (int i = 0; i < t1 - t0; ++i, advance(cur)) {
      const int acc = i & 1;
      // LAST: the residual does not depend on the accumulator: its loads overlap the MMAs
      float res[3] = {0.0f, 0.0f, 0.0f};
      const size_t hw = (size_t)a.H * a.W, off = (size_t)cur.y * a.W + cur.x0 + px;
      if (LAST && h16 == 0 && cur.x0 + px < a.W)
#pragma unroll
        for (int c = 0; c < 3; ++c) res[c] = a.resid[((size_t)cur.b * 3 + c) * hw + off];
      if (!mbar_wait(accf(acc), (i >> 1) & 1, a.spin)) { failed = true; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      uint32_t r[16];
      const uint32_t taddr = tmem + acc * 32 + h16 * 16 + ((uint32_t)(q * 32) << 16);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(acce(acc));
      const int x = cur.x0 + px;
      if (LAST) {  // channels 0-2 of the first half: u0 = f + conv + bias, planar FP32
        if (h16 == 0 && x < a.W)
#pragma unroll
          for (int c = 0; c < 3; ++c)
            a.out_planar[((size_t)cur.b * 3 + c) * hw + off] = (__uint_as_float(r[c]) + sbias[c]) + res[c];
        continue;
      }
      if (x < a.W) {
        const size_t pix = ((size_t)cur.b * a.H + cur.y) * a.W + x;
        uint4 mk[2];
        if (a.mask != nullptr)
#pragma unroll
          for (int t = 0; t < 2; ++t) mk[t] = reinterpret_cast<const uint4*>(a.mask + pix * 32 + h16 * 16)[t];
        uint4 o[2];
        uint32_t* ow = reinterpret_cast<uint32_t*>(o);
#pragma unroll
        for (int c = 0; c < 16; c += 2) {
          const int ch = h16 * 16 + c;
          float v0 = __uint_as_float(r[c]) + sbias[ch], v1 = __uint_as_float(r[c + 1]) + sbias[ch + 1];
          if (a.relu) {
            v0 = fmaxf(v0, 0.0f);
            v1 = fmaxf(v1, 0.0f);
          }
          if (a.mask != nullptr) {
            const __nv_bfloat162 m = reinterpret_cast<const __nv_bfloat162*>(mk)[c >> 1];
            if (!(__bfloat162float(m.x) > 0.0f)) v0 = 0.0f;
            if (!(__bfloat162float(m.y) > 0.0f)) v1 = 0.0f;
          }
          __nv_bfloat162 hv = __floats2bfloat162_rn(v0, v1);
          ow[c >> 1] = *reinterpret_cast<uint32_t*>(&hv);
        }
#pragma unroll
        for (int t = 0; t < 2; ++t) reinterpret_cast<uint4*>(a.out + pix * 32 + h16 * 16)[t] = o[t];
      }
    }
  }
  if (failed) atomicExch(a.error, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem));
}

// ---------------------------------------------------------------- weight gradient
// dW[co][(3 dy + dx) ci_n + ci] += sum_p dY[p][co] X[p + (dy - 1, dx - 1)][ci] and db[co] +=
// sum_p dY[p][co] over every pixel p of the batch: the weight gradient of a conv3x3 with
// ci_n <= 32 input and co_n <= 32 output channels (the 32 -> 32 layers; the 3 -> 32 and
// 32 -> 3 layers with their 3-channel side packed to 8-channel NHWC rows, channels 3-7 zero,
// which the tensor map's zero fill widens to 32).
//
// Written per input row q = p + (dy - 1, 0): the tile of 128 pixels of input row yq contributes
// D[M = (dx, ci)][N = (kb, co)] += sum_x X[yq][x + dx - 1][ci] dY[yq - 1 + kb][x][co], and the
// block kb of N belongs to dy = 2 - kb.  An M = 128 MMA costs about the same whatever its N up
// to 256, so N = 96 (three dY rows) does the work of the three N = 32 products of the dy
// taps in one instruction: 8 MMAs of K = 16 pixels per tile.  Both operands are MN-major in
// the 64-byte swizzled canonical layout, an NHWC row of 32 channels (64 bytes per pixel) as
// TMA writes it with the 64-byte swizzle:
//   A: an input slot holds the tile's input row three times, shifted by dx - 1 pixels, then a
//      block of ones, 8 KB apart: the four 32-row blocks of M are LBO = 8 KB apart, the K
//      groups of 8 pixels SBO = 512 bytes apart.  M rows 96-127 read ones, so row 96 collects
//      sum_p dY[p]: its kb = 1 block (dY row yq itself) is db.
//   B: a ring of dY rows (row r in slot r mod WG_RING) with slots 0 and 1 mirrored after the
//      ring, so rows yq - 1, yq, yq + 1 always sit in three consecutive 8 KB blocks (LBO).
// Each CTA takes a contiguous range of the batch's tiles, ordered by (image, 128-pixel column,
// input row); within a column a tile needs one new dY row.  One thread issues the copies, up
// to WG_XSLOTS tiles ahead: a slot is refilled once the MMAs of its previous tile are done
// (they also were the last to read the dY ring slot the new row takes), and a new column
// starts after every MMA issued is done.  Another thread issues the MMAs of each tile once its
// copies have landed; the two meet only at the mbarriers (with one thread doing both, a
// launch took 48-52 us on the 16 x 256^2 training batch, bound by that thread).  Out-of-image
// pixels come from TMA's zero fill; the input rows -1 and H, which only zero padding would
// pair with, are never walked.  The CTA accumulates its tiles in tensor memory and adds the
// result to dW and db with FP32 atomics at the end.  Every wait is bounded (error flag,
// drain, free), and no mbarrier ever has more than one phase pending.
constexpr int WG_TILE = 128;
constexpr int WG_AHEAD = 3;                            // tiles of copies in flight beyond the current one
constexpr int WG_XSLOTS = WG_AHEAD + 1;                // input slots (also the number of barrier pairs)
constexpr int WG_RING = WG_AHEAD + 3;                  // dY ring slots (+2 mirrors)
constexpr int WG_BLK = WG_TILE * 64;                   // 8192: 128 pixels x 32 BF16 channels
constexpr int WG_XSLOT = 4 * WG_BLK;                   // dx = 0, 1, 2 and the ones block
constexpr int WG_D_BYTES = (WG_RING + 2) * WG_BLK;     // 65536
constexpr int WG_X_BYTES = WG_XSLOTS * WG_XSLOT;       // 131072
constexpr int WG_SMEM = 1024 + WG_D_BYTES + WG_X_BYTES + 2 * WG_XSLOTS * 8;  // + alignment slack
constexpr int WG_NTHR = 128;
// kind::f16 with both operands MN-major (transpose bits 15 and 16), M = 128, N = 96
constexpr uint32_t kIdescWg = tc::idesc_bf16(128, 96) | (1u << 15) | (1u << 16);

struct WgArgs {
  int B, H, W;
  int ci_n, co_n, kpad;  // input and output channels (<= 32), row length of dW
  float* dw;    // [co_n][kpad] FP32, column (3 dy + dx) ci_n + ci (accumulated)
  float* db;    // [co_n] FP32 (accumulated)
  int* error;
  uint32_t spin;
};

__device__ __forceinline__ int wg_ring(int r) { return ((r % WG_RING) + WG_RING) % WG_RING; }

__global__ void __launch_bounds__(WG_NTHR, 1)
conv32_wgrad_tc_kernel(const __grid_constant__ CUtensorMap x_map, const __grid_constant__ CUtensorMap dy_map,
                       WgArgs a) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  // the swizzle pattern repeats every 512 bytes: operands start on a 1024-byte boundary; the dY
  // ring comes first so that every operand address stays inside the two regions
  unsigned char* sD = smraw + ((1024u - (saddr(smraw) & 1023u)) & 1023u);
  unsigned char* sX = sD + WG_D_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sX + WG_X_BYTES);  // full[WG_XSLOTS], done[WG_XSLOTS]
  __shared__ uint32_t tmem_base_slot;
  __shared__ int failed_s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // the ones block of every input slot (the swizzle permutes ones into ones)
  for (int q = threadIdx.x; q < WG_XSLOTS * WG_BLK / 16; q += blockDim.x) {
    const uint32_t one2 = 0x3F803F80u;  // two BF16 1.0
    const int sl = q / (WG_BLK / 16), o = q - sl * (WG_BLK / 16);
    reinterpret_cast<uint4*>(sX + sl * WG_XSLOT + 3 * WG_BLK)[o] = make_uint4(one2, one2, one2, one2);
  }
  if (threadIdx.x == 0) {
    failed_s = 0;
    for (int i = 0; i < 2 * WG_XSLOTS; ++i) mbar_init(saddr(&bars[i]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(saddr(&tmem_base_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_slot;

  const int tiles_x = (a.W + WG_TILE - 1) / WG_TILE;
  const int total = a.B * tiles_x * a.H;  // tile g: column g / H, input row g % H
  const int t0 = (int)((long long)total * blockIdx.x / gridDim.x);
  const int t1 = (int)((long long)total * (blockIdx.x + 1) / gridDim.x);
  // a tile's position (column col of image b at pixel x0, input row yq), advanced one tile at a
  // time: a division only when a column ends
  struct Pos {
    int col, yq, b, x0;
  };
  auto set_col = [&](Pos& p) {
    p.b = p.col / tiles_x;
    p.x0 = (p.col - p.b * tiles_x) * WG_TILE;
  };
  auto start = [&](int g) {
    Pos p;
    p.col = g / a.H;
    p.yq = g - p.col * a.H;
    set_col(p);
    return p;
  };
  auto advance = [&](Pos& p) {
    if (++p.yq == a.H) {
      p.yq = 0;
      ++p.col;
      set_col(p);
    }
  };
  auto full = [&](int j) { return saddr(&bars[j]); };
  auto done = [&](int j) { return saddr(&bars[WG_XSLOTS + j]); };
  auto next_slot = [](int j) { return j + 1 == WG_XSLOTS ? 0 : j + 1; };
  if (warp == 0 && lane == 0 && t1 > t0) {
    // ---------------- copy thread.  Tile g goes to input slot j = (g - t0) mod WG_XSLOTS once the
    // MMAs of the slot's previous tile (g - WG_XSLOTS) are done; those also were the last to read
    // the dY ring slot its new row takes.  A column run starts after every MMA issued is done.
    // Per slot (bit j): loads so far mod 2, a load whose MMAs this thread has not waited for,
    // a slot loaded at least once.
    uint32_t loadpar = 0, outstanding = 0, used = 0;
    bool failed = false;
    // copies for a tile on full[j]: its input row three times, and dY rows yq - 1 .. yq + 1
    // (first tile of a column run) or yq + 1 alone, each into its ring slot and, for slots 0 and
    // 1, the mirror after the ring
    auto load_tile = [&](const Pos& p, int j, bool first) {
      uint32_t bytes = 3 * WG_BLK;
      for (int r = first ? p.yq - 1 : p.yq + 1; r <= p.yq + 1; ++r) bytes += (wg_ring(r) < 2 ? 2 : 1) * WG_BLK;
      mbar_expect_tx(full(j), bytes);
      for (int dx = 0; dx < 3; ++dx)
        tma_load_4d(saddr(sX + j * WG_XSLOT + dx * WG_BLK), &x_map, 0, p.x0 - 1 + dx, p.yq, p.b, full(j));
      for (int r = first ? p.yq - 1 : p.yq + 1; r <= p.yq + 1; ++r) {
        const int sl = wg_ring(r);
        tma_load_4d(saddr(sD + sl * WG_BLK), &dy_map, 0, p.x0, r, p.b, full(j));
        if (sl < 2) tma_load_4d(saddr(sD + (WG_RING + sl) * WG_BLK), &dy_map, 0, p.x0, r, p.b, full(j));
      }
    };
    Pos ld = start(t0);
    int lj = 0;
    for (int g = t0; g < t1 && !failed; ++g) {
      const bool first = g == t0 || ld.yq == 0;
      const uint32_t need = first ? outstanding : (outstanding & (1u << lj));
      for (int sl = 0; sl < WG_XSLOTS; ++sl)
        if ((need >> sl) & 1u) {
          if (!mbar_wait(done(sl), ((loadpar >> sl) & 1u) ^ 1u, a.spin)) {
            failed = true;
            break;
          }
          outstanding &= ~(1u << sl);
        }
      if (failed) break;
      load_tile(ld, lj, first);
      loadpar ^= 1u << lj;
      outstanding |= 1u << lj;
      used |= 1u << lj;
      advance(ld);
      lj = next_slot(lj);
    }
    // every copy issued must have landed before the CTA may end (bounded): the last phase of
    // each slot's full barrier
    for (int sl = 0; sl < WG_XSLOTS; ++sl)
      if (((used >> sl) & 1u) && !mbar_wait(full(sl), ((loadpar >> sl) & 1u) ^ 1u)) failed = true;
    if (failed) failed_s = 1;
  } else if (warp == 1 && lane == 0 && t1 > t0) {
    // ---------------- MMA thread: tile g from input slot j once its copies have landed
    uint32_t fullpar = 0, donebit = 0;
    int lastj = -1;
    bool failed = false;
    Pos cur = start(t0);
    int j = 0;
    for (int g = t0; g < t1; ++g) {
      if (!mbar_wait(full(j), (fullpar >> j) & 1u, a.spin)) {
        failed = true;
        break;
      }
      fullpar ^= 1u << j;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t xa = saddr(sX) + (uint32_t)(j * WG_XSLOT);
      const uint32_t da0 = saddr(sD) + (uint32_t)(wg_ring(cur.yq - 1) * WG_BLK);
#pragma unroll
      for (int ks = 0; ks < WG_TILE / 16; ++ks) {
        // 16 pixels (1 KB) per K step; blocks of 32 M or N LBO = 8 KB apart, K groups SBO = 512 B apart
        const uint64_t da = smem_desc_sw64(xa + ks * 1024, WG_BLK, 512);
        const uint64_t dd = smem_desc_sw64(da0 + ks * 1024, WG_BLK, 512);
        tc::mma_f16(tmem, da, dd, kIdescWg, (g > t0 || ks > 0) ? 1u : 0u);
      }
      mma_commit(done(j));
      donebit ^= 1u << j;
      lastj = j;
      advance(cur);
      j = next_slot(j);
    }
    // the accumulator is complete once the last commit's phase is (MMAs complete in order)
    if (lastj >= 0 && !mbar_wait(done(lastj), ((donebit >> lastj) & 1u) ^ 1u)) failed = true;
    if (failed) failed_s = 1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (failed_s) {
    if (threadIdx.x == 0) atomicExch(a.error, 1);
  } else if (t1 > t0) {
    // thread -> accumulator row m = 32 warp + lane: (dx, ci) = (m / 32, m % 32) for m < 96, m = 96
    // the sums of dY; column block kb holds dy = 2 - kb (db: block kb = 1 of row 96)
    const int m = warp * 32 + lane;
#pragma unroll 1
    for (int kb = 0; kb < 3; ++kb) {
      uint32_t r[32];
      const uint32_t taddr = tmem + kb * 32 + ((uint32_t)(warp * 32) << 16);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
            "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
            "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (m < 96 && (m % 32) < a.ci_n) {
        const int k = ((2 - kb) * 3 + m / 32) * a.ci_n + (m % 32);
#pragma unroll
        for (int co = 0; co < 32; ++co)
          if (co < a.co_n) atomicAdd(&a.dw[co * a.kpad + k], __uint_as_float(r[co]));
      } else if (m == 96 && kb == 1) {
#pragma unroll
        for (int co = 0; co < 32; ++co)
          if (co < a.co_n) atomicAdd(&a.db[co], __uint_as_float(r[co]));
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem));
}

}  // namespace cnn_tc

// ---------------------------------------------------------------- host side

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (fn == nullptr) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

}  // namespace

bool conv32_tc_available() { return encode_fn() != nullptr; }

bool make_nhwc32_map(CUtensorMap* map, const void* act, int B, int H, int W, int box_x, int box_y, int ch) {
  EncodeTiledFn enc = encode_fn();
  if (enc == nullptr || (ch != 8 && ch != 32)) return false;
  // dims (innermost first): channel, x, y, image; box: 8 channels x box_x pixels x box_y rows x 1
  const cuuint64_t px = (cuuint64_t)ch * 2;
  const cuuint64_t dims[4] = {(cuuint64_t)ch, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
  const cuuint64_t strides[3] = {px, (cuuint64_t)W * px, (cuuint64_t)H * W * px};
  const cuuint32_t box[4] = {8, (cuuint32_t)box_x, (cuuint32_t)box_y, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(act), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool make_nhwc32_map_sw64(CUtensorMap* map, const void* act, int B, int H, int W, int box_x, int ch) {
  EncodeTiledFn enc = encode_fn();
  if (enc == nullptr || (ch != 8 && ch != 32)) return false;
  // ch = 8: rows of 8 channels (16 bytes per pixel); the 32-channel box reads channels 8-31
  // as zeros (out of the tensor)
  const cuuint64_t px = (cuuint64_t)ch * 2;
  const cuuint64_t dims[4] = {(cuuint64_t)ch, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
  const cuuint64_t strides[3] = {px, (cuuint64_t)W * px, (cuuint64_t)H * W * px};
  const cuuint32_t box[4] = {32, (cuuint32_t)box_x, 1, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(act), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool make_nhwc8_row_map(CUtensorMap* map, const void* act, int B, int H, int W, int box_px) {
  EncodeTiledFn enc = encode_fn();
  if (enc == nullptr) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)W * 2, (cuuint64_t)H, (cuuint64_t)B};
  const cuuint64_t strides[2] = {(cuuint64_t)W * 16, (cuuint64_t)H * W * 16};
  const cuuint32_t box[3] = {(cuuint32_t)box_px * 2, 1, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<void*>(act), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t conv32_tc_set_attributes() {
  cudaError_t e = cudaFuncSetAttribute(cnn_tc::conv32_ring_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       cnn_tc::SMEM_RING);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(cnn_tc::conv32_ring_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           cnn_tc::SMEM_RING);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(cnn_tc::conv3_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, cnn_tc::SMEM_PIPE_IN8);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(cnn_tc::conv32_wgrad_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              cnn_tc::WG_SMEM);
}

// dW += weight gradient, db += bias gradient of a conv3x3 from its NHWC BF16 input x and
// output gradient dy (B x H x W x x_ch / dy_ch, 32 or 8; channels beyond ci_n / co_n zero); dw
// is [co_n][kpad] FP32 with column (3 dy + dx) ci_n + ci, db [co_n] FP32.  Rows of 8 channels
// are widened to 32 by TMA's zero fill, which costs: a 3-channel side is cheaper in rows of 32
// channels whose channels 3-31 are zero.
cudaError_t launch_wgrad_tc(int B, int H, int W, const void* x, int x_ch, int ci_n, const void* dy, int dy_ch, int co_n,
                            float* dw, int kpad, float* db, int* error, cudaStream_t st) {
  using namespace cnn_tc;
  if (encode_fn() == nullptr) return cudaErrorNotSupported;
  if (ci_n < 1 || ci_n > x_ch || co_n < 1 || co_n > dy_ch || kpad < 9 * ci_n) return cudaErrorInvalidValue;
  CUtensorMap xm, dm;
  if (!make_nhwc32_map_sw64(&xm, x, B, H, W, WG_TILE, x_ch) || !make_nhwc32_map_sw64(&dm, dy, B, H, W, WG_TILE, dy_ch))
    return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long tiles = (long long)B * ((W + WG_TILE - 1) / WG_TILE) * H;
  const int grid = tiles < sms ? (int)tiles : sms;   // one persistent CTA per SM
  WgArgs a{};
  a.B = B; a.H = H; a.W = W;
  a.ci_n = ci_n; a.co_n = co_n; a.kpad = kpad;
  a.dw = dw;
  a.db = db;
  a.error = error;
  const char* spin = getenv("ILS_TEST_TC_SPIN");   // test hook: tiny poll limit -> timeout path
  a.spin = (spin != nullptr && spin[0] != 0) ? (uint32_t)atoi(spin) : kSpinLimit;
  conv32_wgrad_tc_kernel<<<grid, WG_NTHR, WG_SMEM, st>>>(xm, dm, a);
  return cudaGetLastError();
}

namespace {

// out = conv3x3_{cin->32}(in) (+bias, ReLU | mask): in is NHWC BF16 with 32 channels, or
// (in8) 8 channels of which the first 3 are the input
cudaError_t launch_conv_tc(bool in8, int B, int H, int W, const void* in, const void* wt, const float* bias, void* out,
                           const void* mask, int relu, int* error, cudaStream_t st) {
  using namespace cnn_tc;
  if (encode_fn() == nullptr) return cudaErrorNotSupported;
  CUtensorMap map, map2;
  if (in8 ? !make_nhwc8_row_map(&map, in, B, H, W, IN8_C0) || !make_nhwc8_row_map(&map2, in, B, H, W, IN8_C1)
          : !make_nhwc32_map_sw64(&map, in, B, H, W, HALO_W, 32))
    return cudaErrorInvalidValue;
  if (!in8) map2 = map;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int tiles = B * H * ((W + TILE - 1) / TILE);
  const int grid = tiles < 2 * sms ? tiles : 2 * sms;   // two persistent CTAs per SM
  TcArgs a{};
  a.B = B; a.H = H; a.W = W;
  a.wt = static_cast<const bf16*>(wt);
  a.bias = bias;
  a.out = static_cast<bf16*>(out);
  a.mask = static_cast<const bf16*>(mask);
  a.relu = relu;
  a.error = error;
  const char* spin = getenv("ILS_TEST_TC_SPIN");   // test hook: tiny poll limit -> timeout path
  a.spin = (spin != nullptr && spin[0] != 0) ? (uint32_t)atoi(spin) : kSpinLimit;
  if (in8)
    conv3_tc_kernel<<<grid, NTHR, SMEM_PIPE_IN8, st>>>(map, map2, a);
  else
    conv32_ring_tc_kernel<false><<<grid, NTHR, SMEM_RING, st>>>(map, a);
  return cudaGetLastError();
}

}  // namespace

// u0 = f + conv3x3_{32->3}(in) + bias: in NHWC BF16 B x H x W x 32, wt [8][288] BF16 (rows 3-7
// zero), f and u0 planar FP32 B x 3 x H x W.
cudaError_t launch_conv_last_tc(int B, int H, int W, const void* in, const void* wt, const float* bias, const float* f,
                                float* u0, int* error, cudaStream_t st) {
  using namespace cnn_tc;
  if (encode_fn() == nullptr) return cudaErrorNotSupported;
  CUtensorMap map;
  if (!make_nhwc32_map_sw64(&map, in, B, H, W, HALO_W, 32)) return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int tiles = B * H * ((W + TILE - 1) / TILE);
  const int grid = tiles < 2 * sms ? tiles : 2 * sms;
  TcArgs a{};
  a.B = B; a.H = H; a.W = W;
  a.wt = static_cast<const bf16*>(wt);
  a.bias = bias;
  a.out_planar = u0;
  a.resid = f;
  a.error = error;
  const char* spin = getenv("ILS_TEST_TC_SPIN");   // test hook: tiny poll limit -> timeout path
  a.spin = (spin != nullptr && spin[0] != 0) ? (uint32_t)atoi(spin) : kSpinLimit;
  conv32_ring_tc_kernel<true><<<grid, NTHR, SMEM_RING, st>>>(map, a);
  return cudaGetLastError();
}

// out = conv3x3_{32->32}(in) (+bias, ReLU | mask) on NHWC BF16 tensors of B x H x W x 32.
cudaError_t launch_conv32_tc(int B, int H, int W, const void* in, const void* wt, const float* bias, void* out,
                             const void* mask, int relu, int* error, cudaStream_t st) {
  return launch_conv_tc(false, B, H, W, in, wt, bias, out, mask, relu, error, st);
}

// out = conv3x3_{3->32}(in) (+bias, ReLU | mask): in is NHWC BF16 rows of 8 channels (3 values,
// then zeros), wt [32][32] BF16 with column tap * 3 + ci, out NHWC BF16 x 32.
cudaError_t launch_conv3_tc(int B, int H, int W, const void* in8, const void* wt, const float* bias, void* out,
                            const void* mask, int relu, int* error, cudaStream_t st) {
  return launch_conv_tc(true, B, H, W, in8, wt, bias, out, mask, relu, error, st);
}

}  // namespace ils
