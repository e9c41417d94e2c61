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

// One scaled value rounded to nearest even in BF16 (fmt 1) or FP16 (fmt 2): the encode
// kernel's arithmetic.
__device__ __forceinline__ unsigned short float_to_code16(float x, int fmt)
{
    return fmt == 1 ? __bfloat16_as_ushort(__float2bfloat16_rn(x)) : __half_as_ushort(__float2half_rn(x));
}

// Two values to two codes with one paired conversion (each element rounded to nearest
// even, x in the low half): the same bits as two float_to_code16 calls.
template <int FMT>
__device__ __forceinline__ unsigned pack_code2(float2 v)
{
    if constexpr (FMT == 1) {
        const __nv_bfloat162 h = __float22bfloat162_rn(v);
        return *reinterpret_cast<const unsigned *>(&h);
    } else {
        const __half2 h = __float22half2_rn(v);
        return *reinterpret_cast<const unsigned *>(&h);
    }
}

template <int FMT>
__device__ __forceinline__ float2 unpack_code2(unsigned u)
{
    if constexpr (FMT == 1) return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u));
    else return __half22float2(*reinterpret_cast<const __half2 *>(&u));
}

// Four values times the checkpoint's scale s, as codes packed little-endian.
__device__ __forceinline__ uint2 pack_code4(float4 v, int fmt, float s)
{
    const float2 s2 = make_float2(s, s);
    const float2 a = __fmul2_rn(make_float2(v.x, v.y), s2);
    const float2 b = __fmul2_rn(make_float2(v.z, v.w), s2);
    if (fmt == 1) return make_uint2(pack_code2<1>(a), pack_code2<1>(b));
    return make_uint2(pack_code2<2>(a), pack_code2<2>(b));
}

__device__ __forceinline__ float4 unpack_code4(uint2 raw, int fmt, float inv)
{
    float2 a, b;
    if (fmt == 1) {
        a = unpack_code2<1>(raw.x);
        b = unpack_code2<1>(raw.y);
    } else {
        a = unpack_code2<2>(raw.x);
        b = unpack_code2<2>(raw.y);
    }
    const float2 i2 = make_float2(inv, inv);
    a = __fmul2_rn(a, i2);
    b = __fmul2_rn(b, i2);
    return make_float4(a.x, a.y, b.x, b.y);
}

}  // namespace fwi
