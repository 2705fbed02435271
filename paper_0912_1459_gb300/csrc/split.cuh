// Operand splitting of the split-precision tensor-core GEMMs (TF32X3 /
// BF16X3): x = hi + lo with hi rounded to the operand format and lo the
// remainder rounded to the same format.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>
#include <type_traits>

namespace cds {
namespace trc {

// Operand container: FP32 bits for TF32, the 16 bits of a BF16.
template <bool TF32>
using SplitE = std::conditional_t<TF32, float, uint16_t>;

// x = hi + lo with hi rounded to TF32 (round to nearest, ties away from zero,
// on the 13 dropped mantissa bits) and lo the FP32 remainder; the input is
// the float pair (f, r), x = f + r.
__device__ __forceinline__ void split_tf32(float f, float r, float& hi, float& lo) {
    const uint32_t u = (__float_as_uint(f) + 0x1000u) & 0xFFFFE000u;
    hi = __uint_as_float(u);
    lo = (f - hi) + r;   // f - hi is exact (same binade or one apart)
}
__device__ __forceinline__ void split_bf16(float f, float r, uint16_t& hi, uint16_t& lo) {
    const __nv_bfloat16 h = __float2bfloat16_rn(f);
    const __nv_bfloat16 l = __float2bfloat16_rn((f - __bfloat162float(h)) + r);
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(l);
}
template <bool TF32>
__device__ __forceinline__ void split_store(float f, float r, SplitE<TF32>* hi, SplitE<TF32>* lo,
                                            int64_t e) {
    if constexpr (TF32) {
        float h, l;
        split_tf32(f, r, h, l);
        hi[e] = h;
        lo[e] = l;
    } else {
        uint16_t h, l;
        split_bf16(f, r, h, l);
        hi[e] = h;
        lo[e] = l;
    }
}
// x as an FP32 pair (f, r): f = fl(x), r = fl(x - f)
__device__ __forceinline__ void pair_of_double(double x, float& f, float& r) {
    f = (float)x;
    r = (float)(x - (double)f);
}

}  // namespace trc
}  // namespace cds
