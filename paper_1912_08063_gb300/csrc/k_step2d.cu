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
#include <cooperative_groups.h>

#include "code16.cuh"
#include "fwi_internal.h"
#include "step2d_math.cuh"

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

using namespace s2d;

// Global operands of one output row: the row entering the z-queue, the x-window groups
// left and right of the centre, and the pointwise values.
template <int M, bool IMG>
struct RowIn {
    float4 qn, win[2 * (M / 4)], pv, Wv, uv, gv;
};

// Every global load of row z is issued before its arithmetic; with PFR the loads of row
// z + 1 are issued before row z's arithmetic (software pipelining).  STORE (forward only)
// also writes the checkpoint of the input pair (c = u^n, prev = u^{n-1}) in the encode
// kernel's format from the epilogue: the store the schedule asks for right before this
// step, without the encode pass's second read of both fields.
// One CTA's work: x tile bx, z-chunk zc of shot `shot`, from state (cur_base = u^n,
// prev_base = u^{n-1}, overwritten by u^{n+1}) at step n.  p supplies everything else
// (it may live in kernel parameters or in a device table).  With row_tr, the receivers
// are the rn consecutive nodes of row rz from column rx0 on, and the epilogue writes
// their samples u^{n+1} to row_tr[0 .. rn) (forward step only).
template <int M, bool IMG, bool PFR, bool STORE, int PF = 0>
__device__ __forceinline__ void step2d_body(const StepParams &p, const float *cur_base,
                                            float *prev_base, int n, int bx, int shot, int zc,
                                            float *row_tr = nullptr, int rz = -1, int rx0 = 0,
                                            int rn = 0)
{
    constexpr int Q = 2 * M + 1, W4 = M / 4;   // x-window: W4 groups of 4 either side
    const int nz = p.g.nz, nx = p.g.nx, px = p.g.px;
    const int z0 = zc * p.zchunk, z1 = min(nz, z0 + p.zchunk);
    const int x0 = bx * kTile2 + threadIdx.x * 4;
    const bool xin = x0 < nx;
    const int64_t plane = p.g.plane;
    const int64_t sb = (int64_t)shot * p.g.field;
    const float *__restrict__ cur = cur_base + sb;
    float *__restrict__ prev = prev_base + sb;
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
            srcv = p.dt2 * p.wavelet[(int64_t)shot * p.nt + n];
        }
    }
    unsigned mxa = 0u, mxd = 0u;   // bits of max|out| and max|out - c| (p.maxbits set)
    float sca = 1.0f, scd = 1.0f;   // STORE: the checkpoint's scales
    if (STORE && p.st_dtype != 0) {
        sca = p.st_scale[2 * shot];
        scd = p.st_scale[2 * shot + 1];
    }

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

    // PF > 0: the streamed rows PF iterations ahead into L2 (addresses formed from the row
    // each time: pointers carried across iterations cost registers and occupancy)
    for (int z = z0; z < z1; ++z) {
        if (PF > 0 && xin) {
            const int zp = z + PF;
            if (zp + M < nz)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(cur + (int64_t)(zp + M) * plane + x0));
            if (zp < z1) {
                asm volatile("prefetch.global.L2 [%0];" ::"l"(prev + (int64_t)zp * plane + x0));
                if (IMG) {
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(p.gacc + sb + (int64_t)zp * plane + x0));
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(
                        auxb + ((int64_t)zp * plane + x0) * (afmt ? 2 : 4)));
                }
            }
        }
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
        float2 l0, l1;
        lap4<M>(w, q, p.c, l0, l1);
        const float4 c = q[M];
        if (xin) {
            const float4 pv = in.pv, Wv = in.Wv;
            const float4 o = update4(c, l0, l1, pv, Wv, sx, p.sig_z[z],
                                     (!IMG && z == src_z) ? src_e : -1, srcv);
            const float rhs[4] = {o.x, o.y, o.z, o.w};
            *(float4 *)(prev + row + x0) = o;
            if (!IMG && row_tr && z == rz) {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int r = x0 + e - rx0;
                    if (r >= 0 && r < rn) row_tr[r] = rhs[e];
                }
            }
            if (STORE) {
                // FP32 pair unchanged, or 16-bit a = c s_a and d = (c - prev) s_d
                const int64_t ci = (int64_t)shot * p.st_cstride + row + x0;
                if (p.st_dtype == 0) {
                    *(float4 *)((float *)p.st_code + ci) = c;
                    if (p.st_comps == 2) *(float4 *)((float *)p.st_code + ci + p.g.field) = pv;
                } else {
                    unsigned short *cc = (unsigned short *)p.st_code + ci;
                    *(uint2 *)cc = pack_code4(c, p.st_dtype, sca);
                    if (p.st_comps == 2)
                        *(uint2 *)(cc + p.g.field) = pack_code4(
                            make_float4(c.x - pv.x, c.y - pv.y, c.z - pv.z, c.w - pv.w),
                            p.st_dtype, scd);
                }
            }
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

template <int M, bool IMG, bool PFR, bool STORE = false, int PF = 0>
__global__ void __launch_bounds__(kThreads2) k_step2d_reg(const StepParams p)
{
    const int shot = blockIdx.z / p.nzchunks, zc = blockIdx.z - shot * p.nzchunks;
    step2d_body<M, IMG, PFR, STORE, PF>(p, p.cur, p.prev, (p.n_dev ? *p.n_dev : 0) + p.n, blockIdx.x,
                                    shot, zc);
}

// ---- the serving loop's shared launch: one forward step of every request in a table ----

// Step t of a tick for every request of the table: work item w of the persistent loop is
// (x tile, z-chunk) (w - work0) of the entry whose range holds it; the entry's state is
// (u0, u1) at the tick's start, so step t reads u^n from u0 (t even) or u1 (t odd) and
// overwrites the other; entries whose nt ends within the tick skip the steps past it.
template <int M>
__global__ void __launch_bounds__(kThreads2) k_step2d_multi(const Batch2d *__restrict__ tab, int t)
{
    const int count = tab->count, total = tab->total_work;
    int e = 0;
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
        while (e + 1 < count && tab->e[e + 1].work0 <= w) ++e;   // w increases: scan on
        const Batch2dEntry &E = tab->e[e];
        const int n = E.n0 + t;
        if (n >= E.p.nt) continue;
        const int lw = w - E.work0;
        const int bx = lw % E.xtiles, zc = lw / E.xtiles;
        const bool odd = t & 1;
        step2d_body<M, false, true, false>(E.p, odd ? E.u1 : E.u0, odd ? E.u0 : E.u1, n, bx, 0, zc,
                                           E.rec_z >= 0 ? E.traces + (int64_t)n * E.nrec : nullptr,
                                           E.rec_z, E.rec_x0, E.nrec);
    }
}

// The receiver samples of step t, traces[n][r] = u^{n+1}(rec_r), of every entry whose
// step does not sample them itself (nsamp receivers each).
__global__ void k_sample_multi(const Batch2d *__restrict__ tab, int t)
{
    const int count = tab->count, total = tab->total_rec;
    int e = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        while (e + 1 < count && tab->e[e + 1].rec0 <= i) ++e;
        const Batch2dEntry &E = tab->e[e];
        const int n = E.n0 + t;
        if (n >= E.p.nt) continue;
        const int r = i - E.rec0;
        const float *next = (t & 1) ? E.u0 : E.u1;   // the buffer step t wrote
        E.traces[(int64_t)n * E.nrec + r] = next[E.rec_off[r]];
    }
}

// Two forward steps per pass (temporal blocking).  A CTA of 64 threads owns a z-chunk
// [z0, z1) of one shot and a 256-column strip [X0 - M, X0 + 256 - M).  It streams
// t = z0 - M .. z1 + M - 1, computing u^{n+1} at row t on the whole strip (from the u^n
// rows t - M .. t + M in the register queue q0, as the single step does) and u^{n+2} at
// row t - M on the strip's inner 256 - 2M columns [X0, X0 + 256 - 2M).  u^{n+2} takes its
// z-neighbours from a second register queue of u^{n+1} rows, its x-window from a
// shared-memory ring of the last M + 2 u^{n+1} strip rows, and its "prev" u^n from q0's
// oldest entry.  Strips overlap by 2M columns and chunks by 2M rows, so u^{n+1} near a
// strip or chunk edge is computed by both neighbours from the same inputs.  Each CTA
// writes only its inner columns and its own rows, and both new states go to buffers the
// kernel does not read.  Per point and two steps: read u^n, u^{n-1} and W (W twice, the
// second time from L2), and write u^{n+1} and u^{n+2}.  The arithmetic is the single
// step's (lap4, update4), so two blocked steps equal two single steps bit for bit.
template <int M, bool PF>
__global__ void __launch_bounds__(kThreads2) k_step2d_tb2x(const StepParams p, float *out1,
                                                            float *out2)
{
    constexpr int Q = 2 * M + 1, W4 = M / 4, R = M + 2, TW = kTile2 - 2 * M;
    __shared__ float4 ring4[R][kThreads2];
    const int shot = blockIdx.z / p.nzchunks, zc = blockIdx.z - shot * p.nzchunks;
    const int nz = p.g.nz, nx = p.g.nx, px = p.g.px;
    const int z0 = zc * p.zchunk, z1 = min(nz, z0 + p.zchunk);
    const int X0 = blockIdx.x * TW;
    const int t4 = threadIdx.x;
    const int x0 = X0 - M + 4 * t4;                       // this thread's 4 columns
    const bool xg = x0 >= 0 && x0 < nx;                   // inside the grid
    const bool own = t4 >= W4 && t4 < kThreads2 - W4 && x0 < nx;   // u^{n+2} columns
    const int64_t plane = p.g.plane;
    const int64_t sb = (int64_t)shot * p.g.field;
    const float *__restrict__ cur = p.cur + sb;
    const float *__restrict__ prev = p.prev + sb;
    float *__restrict__ o1 = out1 + sb;
    float *__restrict__ o2 = out2 + sb;

    float sx[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) sx[e] = (x0 + e >= 0 && x0 + e < nx) ? p.sig_x[x0 + e] : 0.0f;
    int src_z = -1, src_e = 0;
    float srcv1 = 0.0f, srcv2 = 0.0f;
    if (p.src_off && xg) {
        const int64_t so = p.src_off[shot];
        const int sz = (int)(so / plane), sxx = (int)(so - (int64_t)sz * plane);
        if (sxx >= x0 && sxx < x0 + 4) {
            src_z = sz;
            src_e = sxx - x0;
            const int n = (p.n_dev ? *p.n_dev : 0) + p.n;
            srcv1 = p.dt2 * p.wavelet[(int64_t)shot * p.nt + n];
            srcv2 = p.dt2 * p.wavelet[(int64_t)shot * p.nt + n + 1];
        }
    }
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 q0[Q], q1[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) q1[i] = zero4;
#pragma unroll
    for (int i = 0; i < Q - 1; ++i) {
        const int z = z0 - 2 * M + i;
        q0[i] = ld4(cur, (int64_t)z * plane, x0, px, z >= 0 && z < nz);
    }

    // global operands of iteration t: the u^n row entering q0, level 1's x-window groups,
    // prev and W of row t, and W of row t - M (level 2)
    struct In {
        float4 qn, win[2 * W4], pv, Wv, W2;
    };
    auto load = [&](int t, In &in) {
        const int zn = t + M;
        in.qn = ld4(cur, (int64_t)zn * plane, x0, px, zn >= 0 && zn < nz);
        const bool l1 = t >= 0 && t < nz && xg;
        const int64_t row = (int64_t)t * plane;
#pragma unroll
        for (int j = 0; j < 2 * W4; ++j) {
            const int g4 = j < W4 ? j : j + 1;
            in.win[j] = l1 ? ld4(cur, row, x0 + 4 * (g4 - W4), px, true) : zero4;
        }
        in.pv = l1 ? __ldg((const float4 *)(prev + row + x0)) : zero4;
        in.Wv = l1 ? __ldg((const float4 *)(p.W + row + x0)) : zero4;
        const int zb = t - M;
        in.W2 = (zb >= z0 && zb < z1 && own) ? __ldg((const float4 *)(p.W + (int64_t)zb * plane + x0))
                                             : zero4;
    };
    In nxt;
    if (PF) load(z0 - M, nxt);
    for (int t = z0 - M; t < z1 + M; ++t) {
        In in;
        if (PF) {
            in = nxt;
            if (t + 1 < z1 + M) load(t + 1, nxt);
        } else {
            load(t, in);
        }
        q0[Q - 1] = in.qn;
        float4 v1 = zero4;
        if (t >= 0 && t < nz && xg) {
            const int64_t row = (int64_t)t * plane;
            float w[4 + 2 * M];
#pragma unroll
            for (int g4 = 0; g4 < 2 * W4 + 1; ++g4) {
                const float4 v = (g4 == W4) ? q0[M] : in.win[g4 < W4 ? g4 : g4 - 1];
                w[4 * g4] = v.x, w[4 * g4 + 1] = v.y, w[4 * g4 + 2] = v.z, w[4 * g4 + 3] = v.w;
            }
            float2 l0, l1;
            lap4<M>(w, q0, p.c, l0, l1);
            v1 = update4(q0[M], l0, l1, in.pv, in.Wv, sx, p.sig_z[t], t == src_z ? src_e : -1,
                         srcv1);
            if (own && t >= z0 && t < z1) *(float4 *)(o1 + row + x0) = v1;
        }
        q1[Q - 1] = v1;
        ring4[(t + R) % R][t4] = v1;
        __syncthreads();
        const int zb = t - M;
        if (zb >= z0 && zb < z1 && own) {
            const float4 *rrow = ring4[(zb + R) % R];
            float w[4 + 2 * M];
#pragma unroll
            for (int g4 = 0; g4 < 2 * W4 + 1; ++g4) {
                const float4 v = (g4 == W4) ? q1[M] : rrow[t4 + g4 - W4];
                w[4 * g4] = v.x, w[4 * g4 + 1] = v.y, w[4 * g4 + 2] = v.z, w[4 * g4 + 3] = v.w;
            }
            float2 l0, l1;
            lap4<M>(w, q1, p.c, l0, l1);
            const int64_t row = (int64_t)zb * plane;
            *(float4 *)(o2 + row + x0) = update4(q1[M], l0, l1, q0[0], in.W2, sx, p.sig_z[zb],
                                                 zb == src_z ? src_e : -1, srcv2);
        }
#pragma unroll
        for (int i = 0; i < Q - 1; ++i) {
            q0[i] = q0[i + 1];
            q1[i] = q1[i + 1];
        }
    }
}

template <int M, bool PF>
cudaError_t launch_tb2x(const StepParams &p0, int nshots, float *out1, float *out2,
                        cudaStream_t s)
{
    StepParams p = p0;
    constexpr int TW = kTile2 - 2 * M;
    const int bx = (p.g.nx + TW - 1) / TW;
    const int64_t ctas = (int64_t)bx * nshots;
    static const int resident = [] {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_step2d_tb2x<M, PF>, kThreads2, 0) !=
                cudaSuccess ||
            per < 1) {
            cudaGetLastError();
            per = 1;
        }
        return (sms > 0 ? sms : 152) * per;
    }();
    // z-chunks of at least 8M rows that best fill whole waves; each chunk streams 2M rows
    // of u^{n+1} it does not keep and 2M warm-up rows
    const int maxch = p.g.nz / (8 * M) > 0 ? p.g.nz / (8 * M) : 1;
    int nch = 1;
    double best = -1.0;
    for (int c = 1; c <= maxch && c <= 64; ++c) {
        const int zc = (p.g.nz + c - 1) / c;
        const int64_t cn = (p.g.nz + zc - 1) / zc;
        const int64_t tot = ctas * cn;
        const int64_t waves = (tot + resident - 1) / resident;
        const double fill = (double)tot / ((double)waves * resident);
        const double score = fill / (1.0 + (2.0 * M) / zc);
        if (score > best + 1e-9) {
            best = score;
            nch = (int)cn;
        }
    }
    p.zchunk = (p.g.nz + nch - 1) / nch;
    p.nzchunks = (p.g.nz + p.zchunk - 1) / p.zchunk;
    dim3 grid(bx, 1, p.nzchunks * nshots);
    k_step2d_tb2x<M, PF><<<grid, kThreads2, 0, s>>>(p, out1, out2);
    return cudaGetLastError();
}

// Resident CTAs of one instantiation on the device (registers limit it).
template <int M, bool IMG, bool PFR, bool STORE, int PF>
int resident2()
{
    static const int resident = [] {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_step2d_reg<M, IMG, PFR, STORE, PF>,
                                                          kThreads2, 0) != cudaSuccess ||
            per < 1) {
            cudaGetLastError();
            per = 1;
        }
        return (sms > 0 ? sms : 152) * per;
    }();
    return resident;
}

template <int M, bool IMG>
cudaError_t launch2(const StepParams &p0, int nshots, cudaStream_t s)
{
    StepParams p = p0;
    const int bx = (p.g.nx + kTile2 - 1) / kTile2;
    const int64_t ctas = (int64_t)bx * nshots;
    bool store = false;
    // fields larger than L2 (one field of the launch over 96 MB): the streamed rows are
    // prefetched into L2 ahead of their loads (see below)
    const bool big = (double)p.g.field * 4.0 * nshots > 96.0 * (1 << 20);
    int resident;
    if constexpr (IMG) {
        resident = big ? resident2<M, true, false, false, 1>() : resident2<M, true, false, false, 0>();
    } else {
        store = p.st_code != nullptr;
        resident = store ? (big ? resident2<M, false, true, true, 2>() : resident2<M, false, true, true, 0>())
                         : (big ? resident2<M, false, true, false, 2>() : resident2<M, false, true, false, 0>());
    }
    // z-chunks (at least 4M rows each) that best fill whole waves of resident CTAs; each
    // chunk streams 2M warm-up rows that cost about a third of an output row
    const int maxch = p.g.nz / (4 * M) > 0 ? p.g.nz / (4 * M) : 1;
    int nch = 1;
    double best = -1.0;
    for (int c = 1; c <= maxch && c <= 64; ++c) {
        const int zc = (p.g.nz + c - 1) / c;
        const int64_t cn = (p.g.nz + zc - 1) / zc;
        const int64_t tot = ctas * cn;
        const int64_t waves = (tot + resident - 1) / resident;
        const double fill = (double)tot / ((double)waves * resident);
        const double score = fill / (1.0 + 0.3 * (2.0 * M) / zc);
        if (score > best + 1e-9) {
            best = score;
            nch = (int)cn;
        }
    }
    p.zchunk = (p.g.nz + nch - 1) / nch;
    p.nzchunks = (p.g.nz + p.zchunk - 1) / p.zchunk;
    dim3 grid(bx, 1, p.nzchunks * nshots);
    // prefetch into L2 for fields larger than L2: 2 rows ahead (forward modes) or 1 (reverse);
    // measured on 64 shots of 440 x 1064 (120 MB per field) against none: forward
    // 0.1017 -> 0.0985 ms, forward + store 0.1110 -> 0.108 ms, reverse 0.1582 -> 0.122 ms.
    // Grids that stay in L2 have no DRAM latency for them to hide, so they are off there.
    // forward: row z + 1's loads in flight during row z; reverse (imaging): all of row z's
    // loads first (its pipelined form needs too many registers; measured on 64 shots of
    // 440 x 1064: forward 0.121 -> 0.106 ms, reverse 0.190 -> 0.250 ms)
    if constexpr (IMG) {
        if (big) k_step2d_reg<M, true, false, false, 1><<<grid, kThreads2, 0, s>>>(p);
        else k_step2d_reg<M, true, false, false><<<grid, kThreads2, 0, s>>>(p);
    } else if (store) {
        if (big) k_step2d_reg<M, false, true, true, 2><<<grid, kThreads2, 0, s>>>(p);
        else k_step2d_reg<M, false, true, true><<<grid, kThreads2, 0, s>>>(p);
    } else {
        if (big) k_step2d_reg<M, false, true, false, 2><<<grid, kThreads2, 0, s>>>(p);
        else k_step2d_reg<M, false, true, false><<<grid, kThreads2, 0, s>>>(p);
    }
    return cudaGetLastError();
}

}  // namespace

int step2d_tb2_chunks(const Geom &g, int nshots)
{
    // worth it only when the batch fills the GPU: z-chunks of at least 8M rows, x-strips
    // of 256 - 2M columns, and at least one CTA per SM
    if (g.ndim != 2) return 0;
    const int maxch = g.nz / (8 * g.M);
    const int64_t strips = (g.nx + kTile2 - 2 * g.M - 1) / (kTile2 - 2 * g.M);
    if (maxch < 1 || (int64_t)maxch * strips * nshots < 152) return 0;
    return maxch;
}

cudaError_t launch_step2d_tb2(const StepParams &p, int nshots, float *out1, float *out2,
                              int nchunks, cudaStream_t s)
{
    (void)nchunks;
    // PF (the next row's loads in flight, as in the single step) measured slower here:
    // 283 against 292 Gpts/s on the 64-shot batch
    if (p.g.M == 4) return launch_tb2x<4, false>(p, nshots, out1, out2, s);
    if (p.g.M == 8) return launch_tb2x<8, false>(p, nshots, out1, out2, s);
    return cudaErrorInvalidValue;
}

// ---- temporal blocking on chip: one thread-block cluster per request ----
//
// A small 2-D request is advanced by k steps in one launch.  Its C CTAs (one cluster)
// split the nz rows into bands [r0, r1); each CTA holds its band of u^n and u^{n-1} in
// shared memory for the whole launch, reads the M halo rows above and below from its
// neighbours' shared memory (distributed shared memory of the cluster), and writes
// u^{n+1} over its u^{n-1} band; a cluster barrier separates the steps (hardware, no
// polling).  W, the sponge tables and the wavelet are read from global memory (L2).
// Receivers that form one row are sampled in the epilogue; the source is added by the
// thread owning its node.  The arithmetic of a point is the single step's (lap4,
// update4 on the same operands), so k steps here equal k single steps bit for bit.  The
// states return to global memory at the end of the launch (buffer 0 to u0, 1 to u1, the
// same parity the single steps leave).
constexpr int kClThreads = 512;

template <int M>
__global__ void __launch_bounds__(kClThreads, 1) k_step2d_cluster(const Batch2d *__restrict__ tab, int k)
{
    namespace cg = cooperative_groups;
    constexpr int Q = 2 * M + 1, W4 = M / 4;
    extern __shared__ __align__(16) float smc[];
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    const int req = blockIdx.x / C;   // one cluster per request (uniform per cluster)
    if (req >= tab->count) return;
    const Batch2dEntry &E = tab->e[req];
    const StepParams &p = E.p;
    const int nz = p.g.nz, nx = p.g.nx, px = p.g.px;
    const int r0 = (int)((int64_t)rank * nz / C), r1 = (int)((int64_t)(rank + 1) * nz / C);
    const int rup = rank > 0 ? (int)((int64_t)(rank - 1) * nz / C) : 0;   // first row above
    const int R = r1 - r0, band = (nz + C - 1) / C * px;   // floats per band buffer
    float *b0 = smc, *b1 = smc + band;
    const int G = px / 4;
    for (int i = threadIdx.x; i < R * G; i += blockDim.x) {
        *(float4 *)(b0 + 4 * i) = __ldg((const float4 *)(E.u0 + (int64_t)r0 * px) + i);
        *(float4 *)(b1 + 4 * i) = __ldg((const float4 *)(E.u1 + (int64_t)r0 * px) + i);
    }
    // source node
    int src_z = -1, src_x = -1;
    if (p.src_off) {
        const int64_t so = p.src_off[0];
        src_z = (int)(so / px);
        src_x = (int)(so - (int64_t)src_z * px);
    }
    cl.sync();
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int s = 0; s < k; ++s) {
        const int n = E.n0 + s;
        if (n >= p.nt) break;   // the same for every CTA of the cluster
        const float *cur = (s & 1) ? b1 : b0;
        float *prv = (s & 1) ? b0 : b1;
        const float *up = rank > 0 ? cl.map_shared_rank(cur, rank - 1) : nullptr;
        const float *dn = rank < C - 1 ? cl.map_shared_rank(cur, rank + 1) : nullptr;
        const float srcv = p.dt2 * p.wavelet[n];
        float *row_tr = E.rec_z >= r0 && E.rec_z < r1 ? E.traces + (int64_t)n * E.nrec : nullptr;
        for (int it = threadIdx.x; it < R * G; it += blockDim.x) {
            const int lr = it / G, g = it - lr * G;
            const int z = r0 + lr, x0 = 4 * g;
            if (x0 >= nx) continue;
            float4 q[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int zz = z - M + i;
                const float *src = zz < 0 || zz >= nz ? nullptr
                                   : zz < r0          ? up + (int64_t)(zz - rup) * px
                                   : zz >= r1         ? dn + (int64_t)(zz - r1) * px
                                                      : cur + (int64_t)(zz - r0) * px;
                q[i] = src ? *(const float4 *)(src + x0) : zero4;
            }
            float w[4 + 2 * M];
            const float *rowc = cur + (int64_t)lr * px;
#pragma unroll
            for (int g4 = 0; g4 < 2 * W4 + 1; ++g4) {
                const int xg = x0 + 4 * (g4 - W4);
                const float4 v = g4 == W4 ? q[M] : (xg < 0 || xg >= px ? zero4 : *(const float4 *)(rowc + xg));
                w[4 * g4] = v.x, w[4 * g4 + 1] = v.y, w[4 * g4 + 2] = v.z, w[4 * g4 + 3] = v.w;
            }
            float2 l0, l1;
            lap4<M>(w, q, p.c, l0, l1);
            float sx[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) sx[e] = (x0 + e < nx) ? p.sig_x[x0 + e] : 0.0f;
            const float4 pv = *(const float4 *)(prv + (int64_t)lr * px + x0);
            const float4 Wv = __ldg((const float4 *)(p.W + (int64_t)z * px + x0));
            const int se = (z == src_z && src_x >= x0 && src_x < x0 + 4) ? src_x - x0 : -1;
            const float4 o = update4(q[M], l0, l1, pv, Wv, sx, p.sig_z[z], se, srcv);
            *(float4 *)(prv + (int64_t)lr * px + x0) = o;
            if (row_tr && z == E.rec_z) {
                const float rhs[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int r = x0 + e - E.rec_x0;
                    if (r >= 0 && r < E.nrec) row_tr[r] = rhs[e];
                }
            }
        }
        // every band's u^{n+1} is written and every read of u^n is done
        cl.sync();
    }
    for (int i = threadIdx.x; i < R * G; i += blockDim.x) {
        ((float4 *)(E.u0 + (int64_t)r0 * px))[i] = *(const float4 *)(b0 + 4 * i);
        ((float4 *)(E.u1 + (int64_t)r0 * px))[i] = *(const float4 *)(b1 + 4 * i);
    }
}

int cluster2d_max_smem() { return 220 * 1024; }

int cluster2d_size(int M)
{
    // the largest cluster (16, else 8) of which at least one fits with full shared memory
    const void *fn = M == 8 ? (const void *)k_step2d_cluster<8> : (const void *)k_step2d_cluster<4>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, cluster2d_max_smem()) !=
            cudaSuccess ||
        cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    for (int C : {16, 8}) {
        cudaLaunchConfig_t cfg{};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = C;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(C, 1, 1);
        cfg.blockDim = dim3(kClThreads, 1, 1);
        cfg.dynamicSmemBytes = cluster2d_max_smem();
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nc = 0;
        if (cudaOccupancyMaxActiveClusters(&nc, fn, &cfg) == cudaSuccess && nc > 0) return C;
        cudaGetLastError();
    }
    return 0;
}

cudaError_t launch_step2d_cluster(const Batch2d *tab, int M, int k, int C, int nreq, int smem,
                                  cudaStream_t s)
{
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(C * (nreq > 0 ? nreq : 1), 1, 1);
    cfg.blockDim = dim3(kClThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (M == 4) return cudaLaunchKernelEx(&cfg, k_step2d_cluster<4>, tab, k);
    if (M == 8) return cudaLaunchKernelEx(&cfg, k_step2d_cluster<8>, tab, k);
    return cudaErrorInvalidValue;
}

int multi2d_grid(int M)
{
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per, M == 8 ? (const void *)k_step2d_multi<8> : (const void *)k_step2d_multi<4>,
            kThreads2, 0) != cudaSuccess) {
        cudaGetLastError();
        return 152 * 8;
    }
    return (sms > 0 ? sms : 152) * (per > 0 ? per : 1);
}

cudaError_t launch_step2d_multi(const Batch2d *tab, int M, int t, int grid, cudaStream_t s)
{
    if (M == 4) k_step2d_multi<4><<<grid, kThreads2, 0, s>>>(tab, t);
    else if (M == 8) k_step2d_multi<8><<<grid, kThreads2, 0, s>>>(tab, t);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_sample_multi(const Batch2d *tab, int t, int grid, cudaStream_t s)
{
    k_sample_multi<<<grid, 256, 0, s>>>(tab, t);
    return cudaGetLastError();
}

cudaError_t launch_step2d(const StepParams &p, int nshots, bool imaging, cudaStream_t s)
{
    if (p.g.M == 4) return imaging ? launch2<4, true>(p, nshots, s) : launch2<4, false>(p, nshots, s);
    if (p.g.M == 8) return imaging ? launch2<8, true>(p, nshots, s) : launch2<8, false>(p, nshots, s);
    return cudaErrorInvalidValue;
}

}  // namespace fwi
