// Warp-level TF32 tensor-core helpers of the projected kernels (m16n8k8,
// FP32 accumulation, three-term split for FP32-level accuracy).
#pragma once

#include <stdint.h>

namespace ocd {

// TF32 tensor-core helpers.  A product is carried as three TF32 products
// (hi*hi + hi*lo + lo*hi, the split of Ootomo and Yokota), which keeps the
// result at FP32-level accuracy: hi = x with the 13 low mantissa bits
// cleared (a TF32 value), lo = x - hi (exact in FP32; the tensor core reads
// its leading 19 bits).  Relative error of a split product: about 2^-20.
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = __float_as_uint(x) & 0xffffe000u;
  lo = __float_as_uint(x - __uint_as_float(hi));
}
// D += A B for one m16n8k8 TF32 tile (A row-major 16x8, B column-major 8x8).
// The A fragment here always has a3 == a0 (Re h in both places), so the
// register is passed twice.
__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 "
      "{%0, %1, %2, %3}, {%4, %5, %6, %4}, {%7, %8}, {%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(b0), "r"(b1));
}
// The three split products go to three accumulators (d[0] = hi*hi,
// d[1] = hi*lo, d[2] = lo*hi), so consecutive MMAs of one k-step do not wait
// on each other; they are summed once per pass.
__device__ __forceinline__ void mma3_tf32(float (&d)[3][4], const uint32_t (&ah)[3],
                                          const uint32_t (&al)[3], uint32_t bh0, uint32_t bh1,
                                          uint32_t bl0, uint32_t bl1) {
  mma_tf32(d[0], ah[0], ah[1], ah[2], bh0, bh1);
  mma_tf32(d[1], ah[0], ah[1], ah[2], bl0, bl1);
  mma_tf32(d[2], al[0], al[1], al[2], bh0, bh1);
}

}  // namespace ocd
