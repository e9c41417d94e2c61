// 2-D time step (forward / reverse step with optional imaging) on GB300: register
// z-streaming with L1-served x-windows.
//
// In 2-D a z-plane is a single row of nx points, so a CTA streams along z over rows of a
// 256-wide x tile (64 threads x 4 points).  Each thread keeps the 2M + 1 rows of its four
// points in a register queue (z-neighbours) and reads the x-window of the output row
// (M floats either side, in 16-byte groups) straight from global memory: the row was read
// by the neighbouring threads a few iterations earlier, so those loads hit L1/L2, and the
// kernel needs neither shared memory nor barriers.  prev and W are read once, the new
// row is written once with 16-byte stores: 16 bytes per point per step.  The reverse step
// with imaging (IMG) adds the transposed zero-lag imaging term g += u^m (L mu^{m+1}) with
// the Laplacian it computes for the step (u^m read pointwise, from an FP32 field or in
// place from a 16-bit checkpoint; g read and written: 26-28 bytes per point), and at the
// source point g -= dt^2 w[m] mu^{m+1} / W.  Shots run on grid.z.
#include "code16.cuh"
#include "fwi_internal.h"

namespace fwi {

namespace {

constexpr int kThreads2 = 64;            // threads per CTA
constexpr int kTile2 = 4 * kThreads2;    // x points per CTA

__device__ __forceinline__ float4 ld4(const float *__restrict__ f, int64_t row, int x,
                                      int px, bool zin)
{
    // x is a multiple of 4; groups outside [0, px) and rows outside the grid read as zero
    if (!zin || x < 0 || x >= px) return make_float4(0.f, 0.f, 0.f, 0.f);
    return __ldg((const float4 *)(f + row + x));
}

__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

// Global operands of one output row: the row entering the z-queue, the x-window groups
// left and right of the centre, and the pointwise values.
template <int M, bool IMG>
struct RowIn {
    float4 qn, win[2 * (M / 4)], pv, Wv, uv, gv;
};

// Every global load of row z is issued before its arithmetic; with PFR the loads of row
// z + 1 are issued before row z's arithmetic (software pipelining).
template <int M, bool IMG, bool PFR>
__global__ void __launch_bounds__(kThreads2) k_step2d_reg(const StepParams p)
{
    constexpr int Q = 2 * M + 1, W4 = M / 4;   // x-window: W4 groups of 4 either side
    const int shot = blockIdx.z / p.nzchunks, zc = blockIdx.z - shot * p.nzchunks;
    const int nz = p.g.nz, nx = p.g.nx, px = p.g.px;
    const int z0 = zc * p.zchunk, z1 = min(nz, z0 + p.zchunk);
    const int x0 = blockIdx.x * kTile2 + threadIdx.x * 4;
    const bool xin = x0 < nx;
    const int64_t plane = p.g.plane;
    const int64_t sb = (int64_t)shot * p.g.field;
    const float *__restrict__ cur = p.cur + sb;
    float *__restrict__ prev = p.prev + sb;
    const int afmt = p.aux_fmt;
    const char *__restrict__ auxb =
        IMG ? (const char *)p.aux + (size_t)shot * p.aux_stride * (afmt ? 2 : 4) : nullptr;
    const float ainv = (IMG && p.aux_scale) ? 1.0f / p.aux_scale[2 * shot] : 1.0f;

    float4 q[Q];
#pragma unroll
    for (int i = 0; i < Q - 1; ++i) {
        const int z = z0 - M + i;
        const bool zin = z >= 0 && z < nz;
        q[i] = ld4(cur, (int64_t)z * plane, x0, px, zin);
    }
    float sx[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) sx[e] = (x0 + e < nx) ? p.sig_x[x0 + e] : 0.0f;
    int src_z = -1, src_e = 0;
    float srcv = 0.0f;
    if (p.src_off) {
        const int64_t s = p.src_off[shot];
        const int sz = (int)(s / plane), sxx = (int)(s - (int64_t)sz * plane);
        if (sxx >= x0 && sxx < x0 + 4) {
            src_z = sz;
            src_e = sxx - x0;
            srcv = p.dt2 * p.wavelet[(int64_t)shot * p.nt + (p.n_dev ? *p.n_dev : 0) + p.n];
        }
    }
    const float2 two = make_float2(2.0f, 2.0f);
    unsigned mxa = 0u, mxd = 0u;   // bits of max|out| and max|out - c| (p.maxbits set)

    auto load_row = [&](int z, RowIn<M, IMG> &in) {
        const int zn = z + M;
        const int64_t row = (int64_t)z * plane;
        in.qn = ld4(cur, (int64_t)zn * plane, x0, px, zn < nz);
#pragma unroll
        for (int j = 0; j < 2 * W4; ++j) {
            const int g4 = j < W4 ? j : j + 1;
            in.win[j] = ld4(cur, row, x0 + 4 * (g4 - W4), px, true);
        }
        if (xin) {
            in.pv = __ldg((const float4 *)(prev + row + x0));
            in.Wv = __ldg((const float4 *)(p.W + row + x0));
            if (IMG) {
                in.uv = afmt == 0 ? __ldg((const float4 *)((const float *)auxb + row + x0))
                                  : unpack_code4(__ldg((const uint2 *)((const unsigned short *)auxb +
                                                                       row + x0)),
                                                 afmt, ainv);
                in.gv = *(const float4 *)(p.gacc + sb + row + x0);
            }
        }
    };
    RowIn<M, IMG> nxt;
    if (PFR && z0 < z1) load_row(z0, nxt);

    for (int z = z0; z < z1; ++z) {
        RowIn<M, IMG> in;
        if (PFR) {
            in = nxt;
            if (z + 1 < z1) load_row(z + 1, nxt);
        } else {
            load_row(z, in);
        }
        q[Q - 1] = in.qn;
        const int64_t row = (int64_t)z * plane;
        // x-window of the output row: groups x0 - M .. x0 + 3 + M
        float w[4 + 2 * M];
#pragma unroll
        for (int g4 = 0; g4 < 2 * W4 + 1; ++g4) {
            const float4 v = (g4 == W4) ? q[M] : in.win[g4 < W4 ? g4 : g4 - 1];
            w[4 * g4] = v.x, w[4 * g4 + 1] = v.y, w[4 * g4 + 2] = v.z, w[4 * g4 + 3] = v.w;
        }
        float lx[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float a0 = 0.f, a1 = 0.f;
#pragma unroll
            for (int k = 1; k <= M; ++k) {
                const float s = w[M + e + k] + w[M + e - k];
                if (k & 1) a0 = fmaf(p.c.cx[k], s, a0);
                else a1 = fmaf(p.c.cx[k], s, a1);
            }
            lx[e] = a0 + a1;
        }
        float2 za = make_float2(0.f, 0.f), zb = za;
#pragma unroll
        for (int k = 1; k <= M; ++k) {
            const float2 cc = make_float2(p.c.cz[k], p.c.cz[k]);
            za = __ffma2_rn(cc, __fadd2_rn(lo2(q[M + k]), lo2(q[M - k])), za);
            zb = __ffma2_rn(cc, __fadd2_rn(hi2(q[M + k]), hi2(q[M - k])), zb);
        }
        const float4 c = q[M];
        const float2 c0 = make_float2(p.c.c0, p.c.c0);
        const float2 l0 = __ffma2_rn(c0, lo2(c), __fadd2_rn(za, make_float2(lx[0], lx[1])));
        const float2 l1 = __ffma2_rn(c0, hi2(c), __fadd2_rn(zb, make_float2(lx[2], lx[3])));
        if (xin) {
            const float4 pv = in.pv, Wv = in.Wv;
            const float2 r0 = __ffma2_rn(lo2(Wv), l0, __fmul2_rn(two, lo2(c)));
            const float2 r1 = __ffma2_rn(hi2(Wv), l1, __fmul2_rn(two, hi2(c)));
            float rhs[4] = {r0.x, r0.y, r1.x, r1.y};
            const float pp[4] = {pv.x, pv.y, pv.z, pv.w};
            const float sz = p.sig_z[z];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float s = sx[e] + sz;
                float v = fmaf(s - 1.0f, pp[e], rhs[e]);
                if (!IMG && z == src_z && e == src_e) v += srcv;
                rhs[e] = __fdividef(v, 1.0f + s);
            }
            *(float4 *)(prev + row + x0) = make_float4(rhs[0], rhs[1], rhs[2], rhs[3]);
            if (!IMG && p.maxbits) {
                const float cc[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    mxa = max(mxa, __float_as_uint(rhs[e]) & 0x7fffffffu);
                    mxd = max(mxd, __float_as_uint(rhs[e] - cc[e]) & 0x7fffffffu);
                }
            }
            if (IMG) {
                // g += u^m (L mu^{m+1});  at the source point g -= dt^2 w[m] mu^{m+1} / W
                const float4 uv = in.uv, gv = in.gv;
                float2 g0 = __ffma2_rn(lo2(uv), l0, lo2(gv));
                float2 g1 = __ffma2_rn(hi2(uv), l1, hi2(gv));
                if (z == src_z) {
                    // g[e] -= srcv c[e] / W[e] at the source point e
                    const float ce = src_e == 0 ? c.x : src_e == 1 ? c.y : src_e == 2 ? c.z : c.w;
                    const float we = src_e == 0 ? Wv.x : src_e == 1 ? Wv.y : src_e == 2 ? Wv.z : Wv.w;
                    const float qv = __fdividef(ce, we);
                    if (src_e == 0) g0.x = fmaf(-srcv, qv, g0.x);
                    else if (src_e == 1) g0.y = fmaf(-srcv, qv, g0.y);
                    else if (src_e == 2) g1.x = fmaf(-srcv, qv, g1.x);
                    else g1.y = fmaf(-srcv, qv, g1.y);
                }
                *(float4 *)(p.gacc + sb + row + x0) = make_float4(g0.x, g0.y, g1.x, g1.y);
            }
        }
#pragma unroll
        for (int i = 0; i < Q - 1; ++i) q[i] = q[i + 1];
    }
    if (!IMG && p.maxbits) {
        // the checkpoint codec's max-abs of the new state pair (u^{n+1}, u^n)
        const unsigned a = __reduce_max_sync(0xffffffffu, mxa);
        const unsigned d = __reduce_max_sync(0xffffffffu, mxd);
        if ((threadIdx.x & 31) == 0) {
            if (a) atomicMax(p.maxbits + 2 * shot, a);
            if (d) atomicMax(p.maxbits + 2 * shot + 1, d);
        }
    }
}

template <int M, bool IMG>
cudaError_t launch2(const StepParams &p0, int nshots, cudaStream_t s)
{
    StepParams p = p0;
    const int bx = (p.g.nx + kTile2 - 1) / kTile2;
    const int64_t ctas = (int64_t)bx * nshots;
    // enough CTAs for ~16 resident per SM on 152 SMs, chunks of at least 4M rows
    const int want = (int)((16LL * 152 + ctas - 1) / ctas);
    const int maxch = p.g.nz / (4 * M) > 0 ? p.g.nz / (4 * M) : 1;
    const int nch = want < 1 ? 1 : (want > maxch ? maxch : want);
    p.zchunk = (p.g.nz + nch - 1) / nch;
    p.nzchunks = (p.g.nz + p.zchunk - 1) / p.zchunk;
    dim3 grid(bx, 1, p.nzchunks * nshots);
    // forward: row z + 1's loads in flight during row z; reverse (imaging): all of row z's
    // loads first (its pipelined form needs too many registers; measured on 64 shots of
    // 440 x 1064: forward 0.121 -> 0.106 ms, reverse 0.190 -> 0.250 ms)
    k_step2d_reg<M, IMG, !IMG><<<grid, kThreads2, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_step2d(const StepParams &p, int nshots, bool imaging, cudaStream_t s)
{
    if (p.g.M == 4) return imaging ? launch2<4, true>(p, nshots, s) : launch2<4, false>(p, nshots, s);
    if (p.g.M == 8) return imaging ? launch2<8, true>(p, nshots, s) : launch2<8, false>(p, nshots, s);
    return cudaErrorInvalidValue;
}

}  // namespace fwi
