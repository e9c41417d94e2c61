// Reading checkpoint codes in place: four consecutive 16-bit codes (BF16 or FP16, the
// FWI_SNAP_* types 1 and 2) to FP32, times the reciprocal of the checkpoint's scale.
// Scales are powers of two, so the product equals code / scale exactly: the same values
// the decode kernel (k_aux.cu) writes.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstdint>

namespace fwi {

__device__ __forceinline__ float code16_to_float(unsigned short h, int fmt)
{
    return fmt == 1 ? __bfloat162float(__ushort_as_bfloat16(h)) : __half2float(__ushort_as_half(h));
}

// Four values times the checkpoint's scale, rounded to nearest even in BF16 (fmt 1) or
// FP16 (fmt 2) and packed little-endian: the encode kernel's arithmetic.
__device__ __forceinline__ unsigned short float_to_code16(float x, int fmt)
{
    return fmt == 1 ? __bfloat16_as_ushort(__float2bfloat16_rn(x)) : __half_as_ushort(__float2half_rn(x));
}

__device__ __forceinline__ uint2 pack_code4(float4 v, int fmt, float s)
{
    return make_uint2((unsigned)float_to_code16(v.x * s, fmt) |
                          ((unsigned)float_to_code16(v.y * s, fmt) << 16),
                      (unsigned)float_to_code16(v.z * s, fmt) |
                          ((unsigned)float_to_code16(v.w * s, fmt) << 16));
}

__device__ __forceinline__ float4 unpack_code4(uint2 raw, int fmt, float inv)
{
    return make_float4(code16_to_float((unsigned short)(raw.x & 0xffffu), fmt) * inv,
                       code16_to_float((unsigned short)(raw.x >> 16), fmt) * inv,
                       code16_to_float((unsigned short)(raw.y & 0xffffu), fmt) * inv,
                       code16_to_float((unsigned short)(raw.y >> 16), fmt) * inv);
}

}  // namespace fwi
