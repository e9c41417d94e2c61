// 3-D time step on GB300 (sm_103a): TMA-staged z-streaming stencil (kernel template).
//
// One template serves three modes on the same stencil machinery:
//   kModeStep  out = (2 c + W (L c) - (1 - s) prev [+ dt^2 w[n] at the source]) / (1 + s),
//              written over prev (Eq. 3 with the sponge: the forward step, c = u^n)
//   kModeStepStore  kModeStep that also writes a checkpoint of its input pair (c, prev)
//              in the codec's format from the epilogue (the store the schedule asks for
//              right before this step)
//   kModeAdj   the same update without the source (the reverse step in the W-weighted
//              adjoint variable mu = W nu, c = mu^{m+1}), and the imaging condition
//              g += aux * (L c) with aux = u^m, g -= dt^2 w[m] c / W at the source point;
//              aux is an FP32 field or a 16-bit checkpoint read in place
// where L is the order-2M Laplacian with zero outside the computed grid.  kModeAdj uses
// the transposed form of the zero-lag imaging sum: substituting the forward recursion
// for W L u^m in sum_m mu^{m+1} (L u^m) and the reverse recursion for the result gives
// sum_m u^m (L mu^{m+1}) plus a source-point term (here) and a receiver term (added
// once from the traces), so the reverse step images with the Laplacian it computes
// anyway instead of a second pass over u^m.
//
// A CTA owns a 64 x TY tile of the (x, y) plane and a chunk of z-planes:
//   * one elected thread issues TMA loads (cp.async.bulk.tensor, 4-D maps over
//     [shot][z][y][x]) of the plane's halo tile (64 + 2M) x (TY + 2M) into a ring of
//     SH = M + 1 + P shared-memory stages, and of the pointwise tiles (prev and W, plus
//     aux and g in kModeAdj) into a ring of SP = P + 1 stages; completion is tracked by
//     mbarriers with transaction counts and every wait is bounded;
//   * out-of-grid halo cells are zero-filled by the TMA unit (the Dirichlet condition);
//   * each thread computes 4 (x) x RY (y) points: the z-neighbours come from a register
//     queue of 2M + U planes that shifts by U every U planes (U - 1 spare slots halve or
//     third the register moves), the x/y-neighbours from the resident halo stage of the
//     output plane (it arrived M planes earlier and the ring keeps it);
//   * y and z sums use packed FP32x2 FMAs and split accumulators (independent chains),
//     the x-sums too with option kPackX; the update is prev + increment / (1 + s) in
//     packed form with a fast reciprocal, branch-free; the plane's s_z arrives with its
//     pointwise tiles;
//   * results are stored with 16-byte stores straight from registers.
// Measured on GB300 (radius 8, 512^3): this layout beat a variant that unrolls the
// plane loop so the queue rotates at compile time (larger code, slower), a variant that
// reads the forward z-neighbours from the resident stages instead of registers (more
// shared-memory loads, 15-20 % slower even with the freed registers spent on the options
// below), one thread per 4 x 1 points (16 warps, more y loads, 10 % slower), and
// per-stage release barriers instead of the per-plane CTA barrier (warps drifting a
// plane apart, 16 % slower); U = 2 with packed x-sums beats U = 3 by 1-4 % and U = 1 by
// more than 7 %.
// DRAM traffic per point and step: c once (halo re-reads hit L2), the pointwise fields
// once, the writes once: 16 bytes (kModeStep) or 28 bytes (kModeAdj: + aux, g read and
// written).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <utility>

#include "code16.cuh"
#include "fwi_internal.h"
#include "step3d.h"

namespace fwi {
namespace s3d {

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after `limit` polls, ~2^22 by default (each poll may suspend the
// thread briefly).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int limit = 1 << 22)
{
    for (int i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma_load4(void *dst, const CUtensorMap *map, int x, int y, int z,
                                          int w, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
        : "memory");
}

// Starts bringing the tile of a 4-D tensor map at (x, y, z, w) into L2 (no shared memory,
// no barrier; parts outside the tensor are skipped).
__device__ __forceinline__ void tma_prefetch4(const CUtensorMap *map, int x, int y, int z, int w)
{
    asm volatile("cp.async.bulk.prefetch.tensor.4d.L2.global.tile [%0, {%1, %2, %3, %4}];"
                 ::"l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(w)
                 : "memory");
}

__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

// Approximate reciprocal (PTX rcp.approx), the operation behind the fast division it
// replaces; the damping factor 1 + s lies in [1, 2).
__device__ __forceinline__ float rcp_fast(float d)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
    return r;
}

// max(|a|, |b|) with NaN propagated, as one PTX max; the sign of the result is not
// meaningful (the caller clears it).
__device__ __forceinline__ float absmax_nan(float a, float b)
{
    float r;
    asm("max.NaN.xorsign.abs.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}

// Source-point term of the transposed imaging sum at point e of a 4-point group:
// g[e] -= srcv c[e] / W[e]  (srcv = dt^2 w[m]).
__device__ __forceinline__ void src_image(float2 &g0, float2 &g1, float4 c, float4 W, int e,
                                          float srcv)
{
    const float ce = e == 0 ? c.x : e == 1 ? c.y : e == 2 ? c.z : c.w;
    const float we = e == 0 ? W.x : e == 1 ? W.y : e == 2 ? W.z : W.w;
    const float q = __fdividef(ce, we);
    if (e == 0) g0.x = fmaf(-srcv, q, g0.x);
    else if (e == 1) g0.y = fmaf(-srcv, q, g0.y);
    else if (e == 2) g1.x = fmaf(-srcv, q, g1.x);
    else g1.y = fmaf(-srcv, q, g1.y);
}

// Receivers at output row y, points x0 .. x0 + 3 of plane p.rec_z (p.rec_map set): a
// forward mode writes their samples, the reverse mode adds the residual injection
// inj_scale * q (rounded as the separate injection kernel's atomic add: product, then
// sum) to the new values o before they are stored.
template <int MODE>
__device__ __forceinline__ void rec_epilogue(const Step3dParams &p, int shot, int y, int x0, int nrow,
                                             float (&o)[4])
{
    const int4 ri = __ldg((const int4 *)(p.rec_map + ((int64_t)shot * p.ny + y) * p.px + x0));
    const int idx[4] = {ri.x, ri.y, ri.z, ri.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        if (idx[e] < 0) continue;
        if (MODE != kModeAdj) {
            p.rec_tr[((int64_t)shot * p.nt + nrow) * p.nrec + idx[e]] = o[e];
        } else {
            const float a = p.inj_scale[(int64_t)shot * p.nrec + idx[e]];
            const float q = p.inj_q[((int64_t)shot * p.nt + p.inj_n) * p.nrec + idx[e]];
            o[e] = __fadd_rn(o[e], __fmul_rn(a, q));
        }
    }
}

// Options of the plane loop (bits of Cfg::F):
//   kPackX     x-sums as packed FP32x2 on register pairs that are 64-bit aligned (even
//              offsets pair points (0,1) and (2,3) and add into the y accumulators, odd
//              offsets pair (1,2))
//   kInterior  rows with no damping (s = 0 at all four points) skip the sponge division
//   kIso       isotropic grid (hx = hy = hz): the stencil weights are compile-time
//              constants and the Laplacian is scaled by 1 / h^2 once per point, so the
//              weights take no registers and no loads
constexpr int kPackX = 1, kInterior = 2, kIso = 16;

// Taylor weights of radius M evaluated at compile time from their closed form
// c_k = 2 (-1)^{k+1} (M!)^2 / (k^2 (M-k)! (M+k)!), c_0 = -2 sum_k c_k (the host's
// set-up evaluates the same expression), and the 3-D centre weight 3 c_0.
template <int M>
struct TaylorW {
    float c[M + 1];
    float c0x3;
};

template <int M>
__host__ __device__ constexpr TaylorW<M> taylor_weights()
{
    TaylorW<M> w{};
    double total = 0.0;
    for (int k = 1; k <= M; ++k) {
        double ratio = 1.0;
        for (int i = 1; i <= k; ++i) ratio *= (double)(M - k + i) / (double)(M + i);
        const double ck = ((k & 1) ? 2.0 : -2.0) * ratio / ((double)k * k);
        w.c[k] = (float)ck;
        total += ck;
    }
    w.c[0] = (float)(-2.0 * total);
    w.c0x3 = (float)(-6.0 * total);
    return w;
}

template <int M>
__device__ __forceinline__ float taylor(int k)
{
    constexpr TaylorW<M> w = taylor_weights<M>();
    return w.c[k];
}

template <int M>
__device__ __forceinline__ float taylor_centre3()
{
    constexpr TaylorW<M> w = taylor_weights<M>();
    return w.c0x3;
}

template <int M_, int TY_, int RY_, int P_, int U_, int F_, int NPW_>
struct Cfg {
    static constexpr int M = M_, TY = TY_, RY = RY_, P = P_, U = U_, F = F_;
    static constexpr bool ISO = (F & kIso) != 0;
    static constexpr int NPW = NPW_;   // pointwise tiles per stage
    static constexpr int TX = 64, RX = 4;
    static constexpr int NTX = TX / RX, NTY = TY / RY, NT = NTX * NTY;
    static constexpr int SX = TX + 2 * M, SY = TY + 2 * M;
    static constexpr int SH = M + 1 + P, SP = P + 1, Q = 2 * M + 1;
    // the z-queue holds Q + U - 1 planes and shifts by U every U planes
    static constexpr int L = Q + U - 1;
    static_assert(U >= 1 && U <= 4, "queue shift interval");
    static_assert(M % 2 == 0, "packed x-sums pair even offsets");
    static constexpr int HALO_BYTES = SX * SY * 4;
    static constexpr int TILE_BYTES = TX * TY * 4;
    static constexpr int HALO_STRIDE = (HALO_BYTES + 1023) / 1024 * 1024;
    static constexpr int PW_STRIDE = (NPW * TILE_BYTES + 1023) / 1024 * 1024;
    static constexpr int SMEM = SH * HALO_STRIDE + SP * PW_STRIDE + 1024 /* barriers */ + 1024;
};

// Everything one plane iteration needs; lives in registers (all accesses are inlined).
template <class C, int MODE>
struct Ctx {
    const Step3dParams *p;
    const CUtensorMap *mc, *ma, *mb, *md, *me;
    unsigned char *halo, *pw;
    uint64_t *bar_h, *bar_p;
    int *abort_flag;
    const float *ainv;         // shared: 1 / scale of a 16-bit aux (kModeAdj)
    const float *sts;          // shared: the segment shot's checkpoint scales (st_code)
    float *szs;                // shared: per pointwise stage, sig_z[j & ~3 .. (j & ~3) + 3]
    int tid, tx, ty, za, nout, niter, shot, bx, by, x0, y0, hx, hy;
    int hbase, pbase;         // halo / pointwise loads of the CTA's earlier segments
    int h_issued, p_issued;   // loads issued so far, counted like hbase (thread 0's view)
    float sx1[4], syr[C::RY];  // 1 + sig_x of this thread's columns, sig_y of its rows
    bool xin, sxnz;            // sxnz: some sig_x of this thread's columns is nonzero
    int64_t sb;
    int src_j, src_r, src_e;   // source node in this thread's block (src_j < 0: none)
    float srcv;
    int nrow;                  // step index (the trace row of a forward step)
    float mxa, mxd;            // max|out| and max|out - c| up to sign (p->maxbits set)
    float4 q[C::L][C::RY];

    __device__ __forceinline__ void issue_halo(int it)
    {
        const int st = (hbase + it) % C::SH;
        uint64_t *b = bar_h + st;
        mbar_expect_tx(b, C::HALO_BYTES);
        tma_load4(halo + st * C::HALO_STRIDE, mc, hx, hy, za - C::M + it, shot, b);
    }

    __device__ __forceinline__ void issue_pw(int o)
    {
        const int st = (pbase + o) % C::SP;
        uint64_t *b = bar_p + st;
        unsigned char *d = pw + st * C::PW_STRIDE;
        mbar_expect_tx(b, (C::NPW == 4 && p->aux_fmt != 0 ? 3 * C::TILE_BYTES + C::TILE_BYTES / 2
                                                           : C::NPW * C::TILE_BYTES) + 16);
        // the plane's sponge coefficient rides with its pointwise tiles (16-byte copy of
        // the aligned group of four that holds it; the table is padded past nz)
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], 16, [%2];"
            ::"r"(smem_u32(szs + 4 * st)), "l"(p->sig_z + ((za + o) & ~3)), "r"(smem_u32(b))
            : "memory");
        tma_load4(d, ma, bx * C::TX, by * C::TY, za + o, shot, b);
        tma_load4(d + C::TILE_BYTES, mb, bx * C::TX, by * C::TY, za + o, 0, b);
        if (C::NPW == 4) {
            tma_load4(d + 2 * C::TILE_BYTES, md, bx * C::TX, by * C::TY, za + o, shot, b);
            tma_load4(d + 3 * C::TILE_BYTES, me, bx * C::TX, by * C::TY, za + o, shot, b);
        }
    }

    // One plane iteration `it`; the queue slot of plane (it - 2M + i) is R - 2M + i
    // (R >= 2M), so the newest plane lands in slot R.  Returns false when the loop must
    // stop.
    template <int R>
    __device__ __forceinline__ bool plane(int it)
    {
        constexpr int M = C::M, SX = C::SX, SH = C::SH, SP = C::SP, TX = C::TX, RY = C::RY;
        static_assert(R >= 2 * M && R < C::L, "queue slot");
        if (it >= niter) return false;
        // every thread passes this barrier in every iteration, so an abort raised by any
        // thread in iteration it is seen by all of them here, in iteration it + 1
        __syncthreads();
        if (*(volatile int *)abort_flag) return false;
        if (tid == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            if (it + C::P < niter) {
                issue_halo(it + C::P);
                h_issued = hbase + it + C::P + 1;
            }
            const int op = it - 2 * M + C::P;
            if (op >= 0 && op < nout) {
                issue_pw(op);
                p_issued = pbase + op + 1;
            }
        }
        const int kh = hbase + it;   // this CTA's halo load count
        const int st = kh % SH;
        if (!mbar_wait(bar_h + st, (kh / SH) & 1)) {
            atomicExch(abort_flag, 1);
            return true;
        }
        const float *hk = (const float *)(halo + st * C::HALO_STRIDE);
#pragma unroll
        for (int r = 0; r < RY; ++r)
            q[R][r] = *(const float4 *)(hk + (ty * RY + r + M) * SX + tx * 4 + M);
        if (it < 2 * M) return true;

        const int o = it - 2 * M, j = za + o;
        const int ko = pbase + o;
        const int sp = ko % SP;
        if (!mbar_wait(bar_p + sp, (ko / SP) & 1)) {
            atomicExch(abort_flag, 1);
            return true;
        }
        // the output plane's halo arrived M loads earlier
        const int sj = st >= M ? st - M : st + SH - M;
        const float *hj = (const float *)(halo + sj * C::HALO_STRIDE);
        const float *ta = (const float *)(pw + sp * C::PW_STRIDE);
        const float *tb = ta + TX * C::TY;
        const float sz = szs[4 * sp + (j & 3)];

        // y: rows ty*RY .. ty*RY + 2M + RY - 1 of the halo tile, two accumulators per half
        float2 ya[RY][2], yb[RY][2];
        float4 ctr[RY];
#pragma unroll
        for (int r = 0; r < RY; ++r) ya[r][0] = ya[r][1] = yb[r][0] = yb[r][1] = make_float2(0.f, 0.f);
#pragma unroll
        for (int t = 0; t < 2 * M + RY; ++t) {
            const float4 v = *(const float4 *)(hj + (ty * RY + t) * SX + tx * 4 + M);
#pragma unroll
            for (int r = 0; r < RY; ++r) {
                const int d = t - M - r;
                if (d == 0) {
                    ctr[r] = v;
                } else if (d >= -M && d <= M) {
                    const float2 cc = C::ISO ? make_float2(taylor<M>(d < 0 ? -d : d), taylor<M>(d < 0 ? -d : d))
                                             : p->cy2[d < 0 ? -d : d];
                    if (t & 1) {
                        ya[r][0] = __ffma2_rn(cc, lo2(v), ya[r][0]);
                        ya[r][1] = __ffma2_rn(cc, hi2(v), ya[r][1]);
                    } else {
                        yb[r][0] = __ffma2_rn(cc, lo2(v), yb[r][0]);
                        yb[r][1] = __ffma2_rn(cc, hi2(v), yb[r][1]);
                    }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < RY; ++r) {
            // x window: halo columns tx*4 .. tx*4 + 4 + 2M - 1 of this row
            float w[4 + 2 * M];
            const float *row = hj + (ty * RY + r + M) * SX + tx * 4;
#pragma unroll
            for (int c4 = 0; c4 < (4 + 2 * M) / 4; ++c4) {
                const float4 v = (c4 == M / 4) ? ctr[r] : *(const float4 *)(row + 4 * c4);
                w[4 * c4] = v.x;
                w[4 * c4 + 1] = v.y;
                w[4 * c4 + 2] = v.z;
                w[4 * c4 + 3] = v.w;
            }
            float lx[4];
            if (C::F & kPackX) {
                // offsets k even: the pairs (0,1), (2,3) start at even w indices and add
                // into the y accumulators; k odd: the pair (1,2) does, points 0 and 3 stay
                // scalar
                float2 xm = make_float2(0.f, 0.f);
                float x0 = 0.0f, x3 = 0.0f;
#pragma unroll
                for (int k = 1; k <= M; ++k) {
                    const float ck = C::ISO ? taylor<M>(k) : p->cx[k];
                    const float2 ck2 = make_float2(ck, ck);
                    if ((k & 1) == 0) {
                        ya[r][0] = __ffma2_rn(ck2, __fadd2_rn(make_float2(w[M + k], w[M + k + 1]),
                                                              make_float2(w[M - k], w[M - k + 1])),
                                              ya[r][0]);
                        ya[r][1] = __ffma2_rn(ck2, __fadd2_rn(make_float2(w[M + 2 + k], w[M + 3 + k]),
                                                              make_float2(w[M + 2 - k], w[M + 3 - k])),
                                              ya[r][1]);
                    } else {
                        xm = __ffma2_rn(ck2, __fadd2_rn(make_float2(w[M + 1 + k], w[M + 2 + k]),
                                                        make_float2(w[M + 1 - k], w[M + 2 - k])), xm);
                        x0 = fmaf(ck, w[M + k] + w[M - k], x0);
                        x3 = fmaf(ck, w[M + 3 + k] + w[M + 3 - k], x3);
                    }
                }
                lx[0] = x0;
                lx[1] = xm.x;
                lx[2] = xm.y;
                lx[3] = x3;
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
                    for (int k = 1; k <= M; ++k) {
                        const float s = w[M + e + k] + w[M + e - k];
                        const float ck = C::ISO ? taylor<M>(k) : p->cx[k];
                        if (k & 1) a0 = fmaf(ck, s, a0);
                        else a1 = fmaf(ck, s, a1);
                    }
                    lx[e] = a0 + a1;
                }
            }
            // z from the register queue: plane j +- k sits in slot R - M +- k
            float2 za0 = make_float2(0.f, 0.f), za1 = za0, zb0 = za0, zb1 = za0;
#pragma unroll
            for (int k = 1; k <= M; ++k) {
                const float4 up = q[R - M + k][r], dn = q[R - M - k][r];
                const float2 cc = C::ISO ? make_float2(taylor<M>(k), taylor<M>(k)) : p->cz2[k];
                if (k & 1) {
                    za0 = __ffma2_rn(cc, __fadd2_rn(lo2(up), lo2(dn)), za0);
                    za1 = __ffma2_rn(cc, __fadd2_rn(hi2(up), hi2(dn)), za1);
                } else {
                    zb0 = __ffma2_rn(cc, __fadd2_rn(lo2(up), lo2(dn)), zb0);
                    zb1 = __ffma2_rn(cc, __fadd2_rn(hi2(up), hi2(dn)), zb1);
                }
            }
            const float4 cz4 = q[R - M][r];
            const float2 c0 = C::ISO ? make_float2(taylor_centre3<M>(), taylor_centre3<M>()) : p->c02;
            const float2 s0 = __fadd2_rn(__fadd2_rn(za0, zb0), __fadd2_rn(ya[r][0], yb[r][0]));
            const float2 s1 = __fadd2_rn(__fadd2_rn(za1, zb1), __fadd2_rn(ya[r][1], yb[r][1]));
            float2 l0 = __ffma2_rn(c0, lo2(cz4), __fadd2_rn(s0, make_float2(lx[0], lx[1])));
            float2 l1 = __ffma2_rn(c0, hi2(cz4), __fadd2_rn(s1, make_float2(lx[2], lx[3])));
            if (C::ISO) {
                const float2 ih = make_float2(p->inv_h2, p->inv_h2);
                l0 = __fmul2_rn(l0, ih);
                l1 = __fmul2_rn(l1, ih);
            }

            const int y = y0 + r;
            const int toff = (ty * RY + r) * TX + tx * 4;
            const float4 A = *(const float4 *)(ta + toff);   // prev
            const float4 B = *(const float4 *)(tb + toff);   // W
            const int64_t base = (int64_t)j * p->plane + (int64_t)y * p->px + x0;
            const bool store = xin && y < p->ny;
            const bool at_src = j == src_j && r == src_r;
            // (2c + W lap - (1 - s) prev [+ dt^2 w at the source]) / (1 + s), evaluated as
            // prev + (2 (c - prev) + W lap [+ dt^2 w]) / (1 + s): the division scales only
            // the increment, and 1 + s = (1 + sig_x) + (sig_y + sig_z) pairs up
            const float2 m1 = make_float2(-1.0f, -1.0f), two = make_float2(2.0f, 2.0f);
            const float2 dc0 = __ffma2_rn(lo2(A), m1, lo2(cz4));   // c - prev, exact form
            const float2 dc1 = __ffma2_rn(hi2(A), m1, hi2(cz4));
            float2 t0 = __ffma2_rn(lo2(B), l0, __fmul2_rn(two, dc0));
            float2 t1 = __ffma2_rn(hi2(B), l1, __fmul2_rn(two, dc1));
            if (MODE != kModeAdj && at_src) {
                if (src_e == 0) t0.x += srcv;
                else if (src_e == 1) t0.y += srcv;
                else if (src_e == 2) t1.x += srcv;
                else t1.y += srcv;
            }
            float2 o0, o1;
            if (!(C::F & kInterior) || sxnz || syr[r] != 0.0f || sz != 0.0f) {
                const float syz = syr[r] + sz;
                const float2 d0 = __fadd2_rn(make_float2(sx1[0], sx1[1]), make_float2(syz, syz));
                const float2 d1 = __fadd2_rn(make_float2(sx1[2], sx1[3]), make_float2(syz, syz));
                o0 = __ffma2_rn(t0, make_float2(rcp_fast(d0.x), rcp_fast(d0.y)), lo2(A));
                o1 = __ffma2_rn(t1, make_float2(rcp_fast(d1.x), rcp_fast(d1.y)), hi2(A));
            } else {
                o0 = __fadd2_rn(t0, lo2(A));   // s = 0
                o1 = __fadd2_rn(t1, hi2(A));
            }
            float rhs[4] = {o0.x, o0.y, o1.x, o1.y};
            if (p->rec_map && j == p->rec_z && store) rec_epilogue<MODE>(*p, shot, y, x0, nrow, rhs);
            if (MODE != kModeAdj && p->maxbits) {
                const float cz[4] = {cz4.x, cz4.y, cz4.z, cz4.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    mxa = absmax_nan(mxa, rhs[e]);
                    mxd = absmax_nan(mxd, rhs[e] - cz[e]);
                }
            }
            if (store) *(float4 *)(p->out + sb + base) = make_float4(rhs[0], rhs[1], rhs[2], rhs[3]);
            if (MODE == kModeStepStore && store) {
                // checkpoint of the input pair (c = u^n, prev = u^{n-1}) in the encode
                // kernel's format: FP32 pair, or 16-bit a = c s_a and d = (c - prev) s_d
                const int64_t ci = (int64_t)shot * p->st_cstride + base;
                if (p->st_dtype == 0) {
                    *(float4 *)((float *)p->st_code + ci) = cz4;
                    if (p->st_comps == 2) *(float4 *)((float *)p->st_code + ci + p->field) = A;
                } else {
                    unsigned short *cc = (unsigned short *)p->st_code + ci;
                    *(uint2 *)cc = pack_code4(cz4, p->st_dtype, sts[0]);
                    if (p->st_comps == 2)
                        *(uint2 *)(cc + p->field) =
                            pack_code4(make_float4(dc0.x, dc0.y, dc1.x, dc1.y), p->st_dtype, sts[1]);
                }
            }
            if (MODE == kModeAdj) {
                // g += u^m * (L mu^{m+1});  at the source point g -= dt^2 w[m] mu^{m+1} / W
                const float *td = ta + 2 * TX * C::TY, *te = ta + 3 * TX * C::TY;
                const float4 Ua =
                    p->aux_fmt == 0
                        ? *(const float4 *)(td + toff)
                        : unpack_code4(*(const uint2 *)((const unsigned short *)td + toff),
                                       p->aux_fmt, *ainv);
                const float4 G = *(const float4 *)(te + toff);
                float2 g0 = __ffma2_rn(lo2(Ua), l0, lo2(G));
                float2 g1 = __ffma2_rn(hi2(Ua), l1, hi2(G));
                if (at_src) src_image(g0, g1, cz4, B, src_e, srcv);
                if (store) *(float4 *)(p->g + sb + base) = make_float4(g0.x, g0.y, g1.x, g1.y);
            }
        }
        return true;
    }
};

// Runs planes it .. it + U - 1 of one queue-shift group (newest plane in slot L - U + u).
template <class C, int MODE, int u>
__device__ __forceinline__ bool plane_group(Ctx<C, MODE> &c, int it)
{
    if (!c.template plane<C::L - C::U + u>(it + u)) return false;
    if constexpr (u + 1 < C::U) return plane_group<C, MODE, u + 1>(c, it);
    return true;
}

// Streams output planes z0 .. z1 - 1 of tile column `col` (columns are numbered shot by
// shot, tiles row-major within a shot).  Ring indices continue from the CTA's earlier
// segments (hbase, pbase), so stages and barrier phases stay in step across segments.
template <class C, int MODE>
__device__ __forceinline__ void run_segment(Ctx<C, MODE> &c, int col, int z0, int z1,
                                            int tiles_x, int tiles)
{
    constexpr int M = C::M, RY = C::RY, L = C::L;
    const Step3dParams &p = *c.p;
    c.shot = col / tiles;
    const int tile = col - c.shot * tiles;
    c.bx = tile % tiles_x;
    c.by = tile / tiles_x;
    c.za = z0;
    c.nout = z1 - z0;
    c.niter = c.nout + 2 * M;
    c.x0 = c.bx * C::TX + c.tx * C::RX;
    c.y0 = c.by * C::TY + c.ty * RY;
    c.hx = c.bx * C::TX - M;
    c.hy = c.by * C::TY - M;
#pragma unroll
    for (int e = 0; e < 4; ++e) c.sx1[e] = 1.0f + ((c.x0 + e < p.nx) ? p.sig_x[c.x0 + e] : 0.0f);
    c.sxnz = c.sx1[0] != 1.0f || c.sx1[1] != 1.0f || c.sx1[2] != 1.0f || c.sx1[3] != 1.0f;
#pragma unroll
    for (int r = 0; r < RY; ++r) c.syr[r] = (c.y0 + r < p.ny) ? p.sig_y[c.y0 + r] : 0.0f;
    c.xin = c.x0 < p.nx;
    c.sb = (int64_t)c.shot * p.field;
    c.src_j = -1;
    c.src_r = c.src_e = 0;
    c.srcv = 0.0f;
    c.nrow = (p.n_dev ? *p.n_dev : 0) + p.n;
    if (p.src_off) {
        const int64_t s = p.src_off[c.shot];
        const int sz = (int)(s / p.plane), rem = (int)(s - (int64_t)sz * p.plane);
        const int sy = rem / p.px, sx = rem - sy * p.px;
        if (sy >= c.y0 && sy < c.y0 + RY && sx >= c.x0 && sx < c.x0 + 4) {
            c.src_j = sz;
            c.src_r = sy - c.y0;
            c.src_e = sx - c.x0;
            c.srcv = p.dt2 * p.wavelet[(int64_t)c.shot * p.nt + (p.n_dev ? *p.n_dev : 0) + p.n];
        }
    }
#pragma unroll
    for (int i = 0; i < L; ++i)
#pragma unroll
        for (int r = 0; r < RY; ++r) c.q[i][r] = make_float4(0.f, 0.f, 0.f, 0.f);

    if (c.tid == 0 && MODE == kModeAdj)
        *(float *)c.ainv = p.aux_scale ? 1.0f / p.aux_scale[2 * c.shot] : 1.0f;
    if (c.tid == 0 && MODE == kModeStepStore) {
        ((float *)c.sts)[0] = p.st_scale[2 * c.shot];
        ((float *)c.sts)[1] = p.st_scale[2 * c.shot + 1];
    }
    // every thread is past the previous segment: its stages may be refilled
    __syncthreads();
    if (c.tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        for (int it = 0; it < C::P && it < c.niter; ++it) c.issue_halo(it);
        c.h_issued = c.hbase + (C::P < c.niter ? C::P : c.niter);
    }
    for (int it = 0; it < c.niter; it += C::U) {
        // shift the queue by U: slots L - U .. L - 1 receive the planes of this group
#pragma unroll
        for (int i = 0; i < L - C::U; ++i)
#pragma unroll
            for (int r = 0; r < RY; ++r) c.q[i][r] = c.q[i + C::U][r];
        if (!plane_group<C, MODE, 0>(c, it)) break;
    }
    if (MODE != kModeAdj && p.maxbits) {
        // the codec's maxima of this segment's shot (every thread gets here)
        // magnitudes as bits: unsigned order is magnitude order, NaN above infinity
        const unsigned a = __reduce_max_sync(0xffffffffu, __float_as_uint(c.mxa) & 0x7fffffffu);
        const unsigned d = __reduce_max_sync(0xffffffffu, __float_as_uint(c.mxd) & 0x7fffffffu);
        if ((c.tid & 31) == 0) {
            if (a) atomicMax(p.maxbits + 2 * c.shot, a);
            if (d) atomicMax(p.maxbits + 2 * c.shot + 1, d);
        }
        c.mxa = c.mxd = 0.0f;
    }
    c.hbase += c.niter;
    c.pbase += c.nout;
}

// Walks this CTA's share of the persistent schedule (plan_persistent, schedule_segment):
// seg(col, z0, z1) streams one segment; the walk stops when the CTA's abort flag is
// raised.  Every thread of the CTA takes the same segments.
template <class Seg>
__device__ __forceinline__ void walk_schedule(const Step3dParams &p, int columns, const int *abort_flag,
                                              Seg &&seg)
{
    int col, z0, z1;
    for (int i = 0; schedule_segment(p, columns, (int)blockIdx.x, i, &col, &z0, &z1); ++i) {
        seg(col, z0, z1);
        __syncthreads();
        if (*(volatile const int *)abort_flag) break;
    }
}

// Persistent launch: gridDim.x CTAs.  The first p.rounds rounds give every CTA of
// p.round_ctas one whole tile column (all CTAs stream z in step, so neighbouring tiles'
// halos are read while still in L2); the leftover columns are cut along z into
// p.rem_ctas equal pieces, one per CTA (a piece may end one column and start the next).
template <int M, int TY, int RY, int P, int U, int F, int MODE>
__global__ void __launch_bounds__(Cfg<M, TY, RY, P, U, F, 2>::NT, (M == 4 ? 2 : 1))
k_step3d_tma(const __grid_constant__ Step3dParams p, const __grid_constant__ CUtensorMap map_c,
             const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
             const __grid_constant__ CUtensorMap map_d, const __grid_constant__ CUtensorMap map_e)
{
    using C = Cfg<M, TY, RY, P, U, F, MODE == kModeAdj ? 4 : 2>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // aligned by pointer arithmetic on the shared array (a round trip through an integer
    // would hide the address space, and every shared-memory read would become generic)
    unsigned char *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);

    Ctx<C, MODE> c;
    c.p = &p;
    c.mc = &map_c;
    c.ma = &map_a;
    c.mb = &map_b;
    c.md = &map_d;
    c.me = &map_e;
    c.halo = smem;
    c.pw = smem + C::SH * C::HALO_STRIDE;
    c.bar_h = (uint64_t *)(c.pw + C::SP * C::PW_STRIDE);
    c.bar_p = c.bar_h + C::SH;
    c.abort_flag = (int *)(c.bar_p + C::SP);
    c.ainv = (const float *)(c.abort_flag + 1);
    c.sts = c.ainv + 1;
    c.szs = (float *)((unsigned char *)c.bar_h + 512);
    c.tid = threadIdx.x;
    c.tx = c.tid % C::NTX;
    c.ty = c.tid / C::NTX;
    c.hbase = c.pbase = 0;
    c.h_issued = c.p_issued = 0;
    c.mxa = c.mxd = 0.0f;

    if (c.tid == 0) {
        for (int i = 0; i < C::SH; ++i) mbar_init(c.bar_h + i, 1);
        for (int i = 0; i < C::SP; ++i) mbar_init(c.bar_p + i, 1);
        *c.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }

    const int tiles_x = (p.nx + C::TX - 1) / C::TX;
    const int tiles = tiles_x * ((p.ny + C::TY - 1) / C::TY);
    walk_schedule(p, tiles * p.nshots, c.abort_flag,
                  [&](int col, int z0, int z1) { run_segment(c, col, z0, z1, tiles_x, tiles); });
    __syncthreads();
    if (*(volatile int *)c.abort_flag && c.tid == 0) {
        // a bounded wait gave up: report, then give every copy still in flight (at most the
        // last load of each stage) a bounded chance to land before the CTA's shared memory
        // is released
        atomicOr(p.err, 2u);
        for (int q = c.h_issued - C::SH > 0 ? c.h_issued - C::SH : 0; q < c.h_issued; ++q)
            (void)mbar_wait(c.bar_h + q % C::SH, (q / C::SH) & 1);
        for (int q = c.p_issued - C::SP > 0 ? c.p_issued - C::SP : 0; q < c.p_issued; ++q)
            (void)mbar_wait(c.bar_p + q % C::SP, (q / C::SP) & 1);
    }
}

// Largest prefetch depth <= P whose kModeAdj stages (four pointwise tiles) fit the
// shared memory of the CTAs resident per SM.
template <int M, int TY, int RY, int P, int U, int F>
constexpr int adj_prefetch()
{
    constexpr int budget = (M == 4 ? 232448 / 2 - 1024 : 232448);
    if constexpr (P > 1 && Cfg<M, TY, RY, P, U, F, 4>::SMEM > budget)
        return adj_prefetch<M, TY, RY, P - 1, U, F>();
    return P;
}

// Kernel, block size and dynamic shared memory of one configuration in `mode`.
template <int M, int TY, int RY, int P, int U, int F>
Step3dKernelInfo kernel_info(int mode)
{
    Step3dKernelInfo k;
    if (mode == kModeStep || mode == kModeStepStore) {
        using C = Cfg<M, TY, RY, P, U, F, 2>;
        k.fn = mode == kModeStep ? (Step3dKernel)k_step3d_tma<M, TY, RY, P, U, F, kModeStep>
                                 : (Step3dKernel)k_step3d_tma<M, TY, RY, P, U, F, kModeStepStore>;
        k.threads = C::NT;
        k.smem = C::SMEM;
    } else {
        constexpr int PA = adj_prefetch<M, TY, RY, P, U, F>();
        using C = Cfg<M, TY, RY, PA, U, F, 4>;
        static_assert(C::SMEM <= 232448, "shared memory of the reverse-step kernel");
        k.fn = (Step3dKernel)k_step3d_tma<M, TY, RY, PA, U, F, kModeAdj>;
        k.threads = C::NT;
        k.smem = C::SMEM;
    }
    return k;
}

}  // namespace s3d
}  // namespace fwi
