// 16-bit operand packing of the tensor-memory form's MMA operands
// (PREC 1 = bf16, PREC 2 = fp16): two values per 32-bit word, the element
// with the lower k (or row) index in the low 16 bits, and the rounding used
// for the hi / lo splits.
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

}  // namespace tc
}  // namespace sf
