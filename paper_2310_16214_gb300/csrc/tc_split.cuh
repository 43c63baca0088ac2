// Splitting float32 operands into two 16-bit parts for tensor-core products:
// x = hi + lo with hi the 16-bit rounding of x and lo the 16-bit rounding of
// the remainder x - hi (exact in float32), so that a product accumulated in
// float32 as xh yh + xh yl + xl yh keeps about 22 bits (FP16) or 16 bits
// (BF16) of each operand; the xl yl term lies below the float32 rounding of
// the sum.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "bplg.h"

namespace bplg {

template <int PREC>
struct HiLo;

template <>
struct HiLo<BPLG_TC_BF16> {
    static constexpr uint32_t kFmt = 1;  // instruction-descriptor format of the 16-bit operands
    // (x0, x1) -> packed hi pair and lo pair (x0 in the lower 16 bits)
    static __device__ __forceinline__ void pack(float x0, float x1, uint32_t &hi, uint32_t &lo) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
        hi = *reinterpret_cast<const uint32_t *>(&h);
        lo = *reinterpret_cast<const uint32_t *>(&l);
    }
};

template <>
struct HiLo<BPLG_TC_F16> {
    static constexpr uint32_t kFmt = 0;
    static __device__ __forceinline__ void pack(float x0, float x1, uint32_t &hi, uint32_t &lo) {
        const __half2 h = __floats2half2_rn(x0, x1);
        const float2 hf = __half22float2(h);
        const __half2 l = __floats2half2_rn(x0 - hf.x, x1 - hf.y);
        hi = *reinterpret_cast<const uint32_t *>(&h);
        lo = *reinterpret_cast<const uint32_t *>(&l);
    }
};

}  // namespace bplg
