// Device helpers for the 5th-generation tensor-core kernels (inline PTX): mbarriers with
// bounded waits, TMA tensor loads, shared-memory matrix descriptors, tcgen05.mma (kind::f16,
// BF16 inputs, FP32 accumulator in tensor memory) and its commit.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ils {
namespace tc {

constexpr uint32_t kSpinLimit = 1u << 22;  // polls of a bounded mbarrier wait

__device__ __forceinline__ uint32_t saddr(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait: true when the phase completed, false after `limit` polls
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t limit = kSpinLimit) {
  for (uint32_t i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor: start >> 4 | LBO >> 4 << 16 | SBO >> 4 << 32 | version 1 << 46,
// no swizzle (layout type 0 in bits 61-63).  For the K-major operands used here, LBO is
// the byte distance between the two 8-element K halves of a K = 16 step and SBO the
// distance between consecutive groups of 8 rows (M or N).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// The same descriptor for the 64-byte swizzled canonical layout (swizzle mode 4 in bits
// 61-63): the data as TMA writes it with CU_TENSOR_MAP_SWIZZLE_64B; the start address must
// be 512-byte aligned (matrix base offset 0).  For an MN-major operand LBO is the distance
// between blocks of 32 MN elements and SBO between groups of 8 K rows (64 bytes apart each).
__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return smem_desc(addr, lbo, sbo) | (4ull << 61);
}

// Instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A and B
// (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in bits 17-22,
// M >> 4 in bits 24-28.
constexpr uint32_t idesc_bf16(uint32_t m, uint32_t n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((m >> 4) << 24);
}

// D (tensor memory) (+)= A (smem) x B (smem); accumulate = 0 overwrites D.
__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(tmem_d), "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
}
// the mbarrier completes one phase once all MMAs issued so far by this thread are done
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

}  // namespace tc

// Tensor map of an NHWC BF16 tensor of B x H x W x ch (ch = 32, or 8) with a box of 8 channels
// x box_x pixels x box_y rows x 1 image, zero fill out of bounds (host; false when the driver
// entry point is missing or the encoding fails).
bool make_nhwc32_map(CUtensorMap* map, const void* act, int B, int H, int W, int box_x, int box_y, int ch = 32);
// An NHWC BF16 tensor of B x H x W x ch (ch = 32, or 8) with a box of 32 channels x box_x
// pixels x 1 row, written to shared memory with the 64-byte swizzle (for ch = 8 the box's
// channels 8-31 are the zero fill).
bool make_nhwc32_map_sw64(CUtensorMap* map, const void* act, int B, int H, int W, int box_x, int ch);
// An NHWC BF16 tensor of B x H x W x 8 seen as rows of 8-byte elements (two per pixel), with a
// box of box_px pixels x 1 row x 1 image: one copy moves box_px x 16 contiguous bytes.
bool make_nhwc8_row_map(CUtensorMap* map, const void* act, int B, int H, int W, int box_px);

}  // namespace ils
