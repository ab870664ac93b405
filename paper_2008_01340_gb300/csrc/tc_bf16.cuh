// BF16 tensor-core helpers shared by the BF16 pass and the split form:
// the kind::f16 MMA, its instruction descriptor, the 128-byte-swizzled tile
// addressing and the three-term BF16 split of an FP32 value.
#pragma once

#include "ntt_internal.cuh"

namespace ntt {

// D (TMEM, FP32) [+]= A (smem desc) x B (smem desc), BF16 inputs, one CTA.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Instruction descriptor of kind::f16 with BF16 A and B and FP32 D: D format
// (bits 4-5 = 1), A and B format BF16 (bits 7-9, 10-12 = 1), A / B major (bit
// 15 / 16: 1 = MN-major), N >> 3 (bits 17-22), M >> 4 (bits 24-28).
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, bool a_mn, bool b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn ? 1u : 0u) << 15) | ((b_mn ? 1u : 0u) << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Byte offset of BF16 element (row, col) in a tile of `rows` rows kept as
// 64-column atoms of 128-byte rows, 16-byte chunks swizzled over 8 rows.
__device__ __forceinline__ uint32_t swz(int row, int col, int rows) {
  return (uint32_t)((col >> 6) * rows * 128 + row * 128 + ((((col >> 3) & 7) ^ (row & 7)) << 4) +
                    ((col & 7) << 1));
}

// a = t[0] + t[1] + t[2] with t[i] BF16: t0 = bf16(a), t1 = bf16(a - t0),
// t2 = bf16(a - t0 - t1) (3 x 8 significand bits hold the 24 of FP32).
__device__ __forceinline__ void split3(float a, __nv_bfloat16* t) {
  const __nv_bfloat16 a1 = __float2bfloat16_rn(a);
  const float r1 = a - __bfloat162float(a1);
  const __nv_bfloat16 a2 = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(a2);
  t[0] = a1;
  t[1] = a2;
  t[2] = __float2bfloat16_rn(r2);
}

}  // namespace ntt
