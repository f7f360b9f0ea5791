// Warp-level tensor-core helpers of the mixed-precision fused forward:
// 16-bit operand packing and the m16n8k16 / m16n8k8 MMAs with float32
// accumulation (PREC 1 = bf16 operands, PREC 2 = fp16 operands).
//
// Fragment layouts (per lane, g = lane / 4, t4 = lane % 4):
//  A 16x16 row-major: a0 = (row g, k 2t4..2t4+1), a1 = (row g+8, same k),
//                     a2 = (row g, k 2t4+8..2t4+9), a3 = (row g+8, same k)
//  B 16x8 (k x n):    b0 = (k 2t4..2t4+1, col g), b1 = (k 2t4+8..2t4+9, col g)
//  D 16x8:            d0, d1 = (row g, col 2t4, 2t4+1), d2, d3 = (row g+8, same cols)
//  m16n8k8 uses a0, a1 and b0 only.
// The element with the lower k (or column) index sits in the low 16 bits.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace sf {
namespace tc {

template <int PREC>
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  if constexpr (PREC == 1) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
  } else {
    const __half2 v = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
  }
}

// x after rounding to the 16-bit operand type (for hi / lo splits)
template <int PREC>
__device__ __forceinline__ float round16(float x) {
  if constexpr (PREC == 1)
    return __bfloat162float(__float2bfloat16_rn(x));
  else
    return __half2float(__float2half_rn(x));
}

template <int PREC>
__device__ __forceinline__ void mma16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  if constexpr (PREC == 1)
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  else
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int PREC>
__device__ __forceinline__ void mma8(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t b0) {
  if constexpr (PREC == 1)
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(b0));
  else
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(b0));
}

}  // namespace tc
}  // namespace sf
