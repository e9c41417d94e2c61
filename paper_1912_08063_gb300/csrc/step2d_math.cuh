// Arithmetic of one 2-D step on a group of 4 points (shared by every 2-D step kernel, so
// all of them give the same results bit for bit): the order-2M Laplacian from an x-window
// and a z-queue, and the damped leapfrog update.
#pragma once

#include <cuda_runtime.h>

#include "fwi_internal.h"

namespace fwi {
namespace s2d {

__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

// L c at the 4 points of a group: x from the window w (groups x0 - M .. x0 + 3 + M, the
// centre group at w[M .. M + 3]), z from the queue q (row j + k in q[M + k]).
template <int M>
__device__ __forceinline__ void lap4(const float (&w)[4 + 2 * M], const float4 (&q)[2 * M + 1],
                                     const Coefs &cf, float2 &l0, float2 &l1)
{
    float lx[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        float a0 = 0.f, a1 = 0.f;
#pragma unroll
        for (int k = 1; k <= M; ++k) {
            const float s = w[M + e + k] + w[M + e - k];
            if (k & 1) a0 = fmaf(cf.cx[k], s, a0);
            else a1 = fmaf(cf.cx[k], s, a1);
        }
        lx[e] = a0 + a1;
    }
    float2 za = make_float2(0.f, 0.f), zb = za;
#pragma unroll
    for (int k = 1; k <= M; ++k) {
        const float2 cc = make_float2(cf.cz[k], cf.cz[k]);
        za = __ffma2_rn(cc, __fadd2_rn(lo2(q[M + k]), lo2(q[M - k])), za);
        zb = __ffma2_rn(cc, __fadd2_rn(hi2(q[M + k]), hi2(q[M - k])), zb);
    }
    const float4 c = q[M];
    const float2 c0 = make_float2(cf.c0, cf.c0);
    l0 = __ffma2_rn(c0, lo2(c), __fadd2_rn(za, make_float2(lx[0], lx[1])));
    l1 = __ffma2_rn(c0, hi2(c), __fadd2_rn(zb, make_float2(lx[2], lx[3])));
}

// The damped update of a group: (2c + W lap - (1 - s) prev [+ srcv at point se]) / (1 + s).
__device__ __forceinline__ float4 update4(float4 c, float2 l0, float2 l1, float4 pv, float4 Wv,
                                          const float (&sx)[4], float sz, int se, float srcv)
{
    const float2 two = make_float2(2.0f, 2.0f);
    const float2 r0 = __ffma2_rn(lo2(Wv), l0, __fmul2_rn(two, lo2(c)));
    const float2 r1 = __ffma2_rn(hi2(Wv), l1, __fmul2_rn(two, hi2(c)));
    float rhs[4] = {r0.x, r0.y, r1.x, r1.y};
    const float pp[4] = {pv.x, pv.y, pv.z, pv.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const float s = sx[e] + sz;
        float v = fmaf(s - 1.0f, pp[e], rhs[e]);
        if (e == se) v += srcv;
        rhs[e] = __fdividef(v, 1.0f + s);
    }
    return make_float4(rhs[0], rhs[1], rhs[2], rhs[3]);
}

}  // namespace s2d
}  // namespace fwi
