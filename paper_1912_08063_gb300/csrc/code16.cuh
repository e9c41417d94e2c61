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

__device__ __forceinline__ float4 unpack_code4(uint2 raw, int fmt, float inv)
{
    return make_float4(code16_to_float((unsigned short)(raw.x & 0xffffu), fmt) * inv,
                       code16_to_float((unsigned short)(raw.x >> 16), fmt) * inv,
                       code16_to_float((unsigned short)(raw.y & 0xffffu), fmt) * inv,
                       code16_to_float((unsigned short)(raw.y >> 16), fmt) * inv);
}

}  // namespace fwi
