// 3-D time step on GB300 (sm_103a), radius 8 and 4: the z-stream held in tensor memory.
//
// Same three modes and the same arithmetic contract as k_step3d.cuh (kModeStep,
// kModeStepStore, kModeAdj; Eq. 3 with the sponge, the W-weighted reverse step and the
// transposed imaging term), with a data flow built for two CTAs per SM:
//
//   * the x- and y-parts of the Laplacian of a plane are computed when that plane's
//     halo tile arrives (TMA into a ring of only P + 1 shared-memory stages: a halo
//     stage is consumed in the iteration it lands in, not M planes later);
//   * the z-part is split in two halves (a semi-stencil): when plane i arrives, its
//     partial  P(i) = Lxy(i) + c0 u(i) + sum_k c_k u(i - k)  (the past half) is formed
//     from the planes already streamed, and the output plane j = i - M is finished as
//     L(j) = P(j) + sum_k c_k u(j + k)  (the future half, planes j + 1 .. i);
//   * the planes i - M .. i - 1 of u and the partials P(i - M) .. P(i - 1) live in two
//     rings of M slots in tensor memory (TMEM, 32 M columns per CTA, 16 M per thread:
//     each thread owns one TMEM lane and 8 values per slot), read with tcgen05.ld and
//     written with tcgen05.st at addresses computed from the plane index, so the queue
//     never moves between registers;
//   * the update and the epilogue of plane j (prev and W, and u^m and g in kModeAdj,
//     arrive as TMA tiles) are those of k_step3d.cuh.
// With the register queue gone a thread needs at most 128 registers, and with the short
// halo ring a CTA needs ~96 KB (forward) or ~110 KB (reverse) of shared memory, so two
// CTAs (16 warps) share an SM where the register-queue kernel fits one (8 warps).
// DRAM traffic per point and step is unchanged: 16 bytes (kModeStep), 18 with the
// checkpoint store, 26 or 28 in kModeAdj.
//
// TMEM: warp w reads and writes lanes 32 (w mod 4) .. 32 (w mod 4) + 31 (the lane
// quarter the hardware gives it) and columns 16 M (w / 4) .. 16 M (w / 4) + 16 M - 1 of
// its CTA's allocation: raw ring at the first 8 M of those (slot s = plane mod M at 8 s),
// partial ring at the next 8 M.  Allocation is made by warp 0 at the start and released
// by warp 0 at the end, on every path (including a bounded wait that gave up).  An SM
// holds at most two CTAs of these kernels (their shared memory sees to that), and their
// allocations (256 columns each at radius 8, 128 at radius 4) fit its 512, so an
// allocation never waits.
#pragma once

#include "k_step3d.cuh"

namespace fwi {
namespace s3tm {

using s3d::absmax_nan;
using s3d::hi2;
using s3d::lo2;
using s3d::mbar_expect_tx;
using s3d::mbar_init;
using s3d::mbar_try_wait;
using s3d::mbar_wait;
using s3d::rcp_fast;
using s3d::smem_u32;
using s3d::src_image;
using s3d::tma_prefetch4;
using s3d::taylor;
using s3d::taylor_centre3;
using s3d::tma_load4;
constexpr int kPackX = s3d::kPackX, kIso = s3d::kIso;
// Reverse step: each thread copies its own g values of the plane into a shared buffer
// with cp.async at the top of the plane (the tile itself brought into L2 one plane
// earlier), instead of g as a fourth TMA pointwise tile
constexpr int kGAsync = 32;
// Forward modes: 64 x 16 tiles of 4 warps, four CTAs per SM (the same 16 warps and the
// same 512 TMEM columns as two CTAs of 8 warps, with a barrier per 4 warps per plane)
constexpr int kHalf = 64;
template <bool B> struct BoolC { static constexpr bool value = B; };

// ---- tensor memory (tcgen05) ----

__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t cols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(dst)),
                 "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t cols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols)
                 : "memory");
}

__device__ __forceinline__ void tmem_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 8 consecutive columns of this thread's lane.
__device__ __forceinline__ void tmem_st8(uint32_t taddr, float4 a, float4 b)
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
        "r"(__float_as_uint(a.x)), "r"(__float_as_uint(a.y)), "r"(__float_as_uint(a.z)),
        "r"(__float_as_uint(a.w)), "r"(__float_as_uint(b.x)), "r"(__float_as_uint(b.y)),
        "r"(__float_as_uint(b.z)), "r"(__float_as_uint(b.w))
        : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Four slots of 8 columns each (addresses t0..t3) loaded and waited for in one statement,
// so no use of the results can be scheduled before the wait.
struct Slot8 {
    float4 a, b;   // points (row 0, x 0..3), (row 1, x 0..3)
};

#define FWI_TM_OUT8(v) "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])

__device__ __forceinline__ void tmem_ld4x8(uint32_t t0, uint32_t t1, uint32_t t2, uint32_t t3, Slot8 &s0,
                                           Slot8 &s1, Slot8 &s2, Slot8 &s3)
{
    uint32_t r0[8], r1[8], r2[8], r3[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%32];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8, %9, %10, %11, %12, %13, %14, %15}, [%33];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16, %17, %18, %19, %20, %21, %22, %23}, [%34];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%24, %25, %26, %27, %28, %29, %30, %31}, [%35];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : FWI_TM_OUT8(r0), FWI_TM_OUT8(r1), FWI_TM_OUT8(r2), FWI_TM_OUT8(r3)
        : "r"(t0), "r"(t1), "r"(t2), "r"(t3)
        : "memory");
    s0.a = make_float4(__uint_as_float(r0[0]), __uint_as_float(r0[1]), __uint_as_float(r0[2]), __uint_as_float(r0[3]));
    s0.b = make_float4(__uint_as_float(r0[4]), __uint_as_float(r0[5]), __uint_as_float(r0[6]), __uint_as_float(r0[7]));
    s1.a = make_float4(__uint_as_float(r1[0]), __uint_as_float(r1[1]), __uint_as_float(r1[2]), __uint_as_float(r1[3]));
    s1.b = make_float4(__uint_as_float(r1[4]), __uint_as_float(r1[5]), __uint_as_float(r1[6]), __uint_as_float(r1[7]));
    s2.a = make_float4(__uint_as_float(r2[0]), __uint_as_float(r2[1]), __uint_as_float(r2[2]), __uint_as_float(r2[3]));
    s2.b = make_float4(__uint_as_float(r2[4]), __uint_as_float(r2[5]), __uint_as_float(r2[6]), __uint_as_float(r2[7]));
    s3.a = make_float4(__uint_as_float(r3[0]), __uint_as_float(r3[1]), __uint_as_float(r3[2]), __uint_as_float(r3[3]));
    s3.b = make_float4(__uint_as_float(r3[4]), __uint_as_float(r3[5]), __uint_as_float(r3[6]), __uint_as_float(r3[7]));
}
__device__ __forceinline__ void tmem_ld5x8(uint32_t t0, uint32_t t1, uint32_t t2, uint32_t t3, uint32_t t4,
                                           Slot8 &s0, Slot8 &s1, Slot8 &s2, Slot8 &s3, Slot8 &s4)
{
    uint32_t r0[8], r1[8], r2[8], r3[8], r4[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%40];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8, %9, %10, %11, %12, %13, %14, %15}, [%41];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16, %17, %18, %19, %20, %21, %22, %23}, [%42];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%24, %25, %26, %27, %28, %29, %30, %31}, [%43];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%32, %33, %34, %35, %36, %37, %38, %39}, [%44];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : FWI_TM_OUT8(r0), FWI_TM_OUT8(r1), FWI_TM_OUT8(r2), FWI_TM_OUT8(r3), FWI_TM_OUT8(r4)
        : "r"(t0), "r"(t1), "r"(t2), "r"(t3), "r"(t4)
        : "memory");
    uint32_t *rr[5] = {r0, r1, r2, r3, r4};
    Slot8 *ss[5] = {&s0, &s1, &s2, &s3, &s4};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        ss[k]->a = make_float4(__uint_as_float(rr[k][0]), __uint_as_float(rr[k][1]),
                               __uint_as_float(rr[k][2]), __uint_as_float(rr[k][3]));
        ss[k]->b = make_float4(__uint_as_float(rr[k][4]), __uint_as_float(rr[k][5]),
                               __uint_as_float(rr[k][6]), __uint_as_float(rr[k][7]));
    }
}
#undef FWI_TM_OUT8

// acc += c * v on both packed halves of a 4-point row
__device__ __forceinline__ void fma4(float2 &lo, float2 &hi, float c, float4 v)
{
    const float2 c2 = make_float2(c, c);
    lo = __ffma2_rn(c2, lo2(v), lo);
    hi = __ffma2_rn(c2, hi2(v), hi);
}

// M: radius (8).  P: halo prefetch depth (halo ring of P + 1 stages).  PP: pointwise
// prefetch depth (ring of PP + 1 stages).  F: option bits (kPackX, kIso).  NPW: pointwise
// tiles per stage (2: prev, W; 4: + u^m, g).
template <int M_, int P_, int PP_, int F_, int NPW_>
struct Cfg {
    static constexpr int M = M_, P = P_, PP = PP_, F = F_, NPW = NPW_;
    static constexpr bool ISO = (F & kIso) != 0;
    static constexpr int TX = 64, TY = (F & kHalf) ? 16 : 32, RX = 4, RY = 2;
    static constexpr int NTX = TX / RX, NTY = TY / RY, NT = NTX * NTY;
    static constexpr int SX = TX + 2 * M, SY = TY + 2 * M;
    static constexpr int SH = P + 1, SP = PP + 1;
    static_assert(M == 8 || M == 4, "the TMEM rings hold M slots (plane mod M)");
    static constexpr uint32_t RING = 8u * M;   // columns of one ring
    static_assert((NT == 256 || NT == 128) && RX * RY == 8, "8 values per TMEM slot, 4 or 8 warps");
    // TMEM columns per CTA: the raw and partial rings of each warp that shares a lane quarter
    static constexpr uint32_t TCOLS = 2u * RING * (uint32_t)(NT / 128);
    static constexpr int HALO_BYTES = SX * SY * 4;
    static constexpr int TILE_BYTES = TX * TY * 4;
    static constexpr int HALO_STRIDE = (HALO_BYTES + 127) / 128 * 128;
    static constexpr int PW_STRIDE = (NPW * TILE_BYTES + 127) / 128 * 128;
    static constexpr int MISC = 256;   // barriers, flags, scales, sponge groups, TMEM base
    static constexpr int GS = (F & kGAsync) ? 1 : 0;   // g staging buffer
    static constexpr int SMEM = SH * HALO_STRIDE + SP * PW_STRIDE + GS * TILE_BYTES + MISC + 1024;
    // the CTAs that shared memory admits per SM never need more TMEM than the SM's 512
    // columns, so an allocation never waits
    static_assert((233472 / (SMEM + 1024)) * TCOLS <= 512, "a CTA would wait for TMEM");
    static_assert(2 * (SMEM + 1024) <= 233472, "two CTAs per SM");
};

template <class C, int MODE>
struct Ctx {
    const Step3dParams *p;
    const CUtensorMap *mc, *ma, *mb, *md, *me;
    unsigned char *halo, *pw;
    float *gbuf;
    uint64_t *bar_h, *bar_p;
    int *abort_flag;
    const float *ainv;
    const float *sts;
    float *szs;
    uint32_t traw, tpart;       // TMEM addresses of this thread's rings (slot 0)
    int tid, tx, ty, za, nout, niter, shot, bx, by, x0, y0, hx, hy;
    // ring positions: the next halo / pointwise stage to consume (with its phase bit) and
    // to fill (thread 0), and the loads issued so far (for the drain after an abort)
    int hst, hph, pst, pph, hfill, pfill, h_issued, p_issued;
    float sx1[4], syr[C::RY];
    bool rowok[C::RY];          // this thread's rows r store (inside the grid)
    int64_t plane_f;            // floats per z-plane
    float *outp;                // out at (plane 0, row y0, column x0) of this shot
    float *gp;                  // kModeAdj: g at the same place
    unsigned short *codep;      // kModeStepStore with 16-bit codes: code at the same place
    float *codef;               // kModeStepStore with FP32: the same
    int src_j, src_r, src_e;   // source node in this thread's block (src_j < 0: none)
    int src_z;                  // the source node's plane in this shot (-1: none)
    float srcv;
    int nrow;                  // step index (the trace row of a forward step)
    bool domax;                 // raise the checkpoint maxima (p->maxbits set)
    float mxa, mxd;

    __device__ __forceinline__ void issue_halo(int it)
    {
        uint64_t *b = bar_h + hfill;
        mbar_expect_tx(b, C::HALO_BYTES);
        tma_load4(halo + hfill * C::HALO_STRIDE, mc, hx, hy, za - C::M + it, shot, b);
        hfill = hfill + 1 == C::SH ? 0 : hfill + 1;
        ++h_issued;
    }

    __device__ __forceinline__ void issue_pw(int o)
    {
        const int st = pfill;
        uint64_t *b = bar_p + st;
        unsigned char *d = pw + st * C::PW_STRIDE;
        mbar_expect_tx(b, (C::NPW >= 3 && p->aux_fmt != 0 ? (C::NPW - 1) * C::TILE_BYTES + C::TILE_BYTES / 2
                                                           : C::NPW * C::TILE_BYTES) + 16);
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], 16, [%2];"
            ::"r"(smem_u32(szs + 4 * st)), "l"(p->sig_z + ((za + o) & ~3)), "r"(smem_u32(b))
            : "memory");
        tma_load4(d, ma, bx * C::TX, by * C::TY, za + o, shot, b);
        tma_load4(d + C::TILE_BYTES, mb, bx * C::TX, by * C::TY, za + o, 0, b);
        if (C::NPW >= 3) tma_load4(d + 2 * C::TILE_BYTES, md, bx * C::TX, by * C::TY, za + o, shot, b);
        if (C::NPW == 4) tma_load4(d + 3 * C::TILE_BYTES, me, bx * C::TX, by * C::TY, za + o, shot, b);
        pfill = pfill + 1 == C::SP ? 0 : pfill + 1;
        ++p_issued;
    }

    // A bounded wait whose outcome every lane of the warp shares (the TMEM instructions
    // that follow are warp-collective, so no lane may skip them alone).
    // Forward modes probe once before the polling loop (552^3: forward 0.535 -> 0.521 ms,
    // forward + store 0.600 -> 0.579 ms; no gain for the reverse step).
    __device__ __forceinline__ bool wait_warp(uint64_t *bar, uint32_t parity)
    {
        if (MODE != kModeAdj && __all_sync(0xffffffffu, mbar_try_wait(bar, parity))) return true;
        return __all_sync(0xffffffffu, mbar_wait(bar, parity));
    }

    // Lxy(i) + c0 u(i) of this thread's 8 points from the halo tile hk of plane i; also
    // returns u(i) (the tile's centre values).
    __device__ __forceinline__ void lap_xy(const float *hk, float2 (&acc)[C::RY][2], float4 (&ctr)[C::RY])
    {
        constexpr int M = C::M, SX = C::SX, RY = C::RY;
        float2 ya[RY][2], yb[RY][2];
#pragma unroll
        for (int r = 0; r < RY; ++r) ya[r][0] = ya[r][1] = yb[r][0] = yb[r][1] = make_float2(0.f, 0.f);
#pragma unroll
        for (int t = 0; t < 2 * M + RY; ++t) {
            const float4 v = *(const float4 *)(hk + (ty * RY + t) * SX + tx * 4 + M);
#pragma unroll
            for (int r = 0; r < RY; ++r) {
                const int d = t - M - r;
                if (d == 0) {
                    ctr[r] = v;
                } else if (d >= -M && d <= M) {
                    const int ad = d < 0 ? -d : d;
                    const float2 cc = C::ISO ? make_float2(taylor<M>(ad), taylor<M>(ad)) : p->cy2[ad];
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
            float w[4 + 2 * M];
            const float *row = hk + (ty * RY + r + M) * SX + tx * 4;
#pragma unroll
            for (int c4 = 0; c4 < (4 + 2 * M) / 4; ++c4) {
                const float4 v = (c4 == M / 4) ? ctr[r] : *(const float4 *)(row + 4 * c4);
                w[4 * c4] = v.x;
                w[4 * c4 + 1] = v.y;
                w[4 * c4 + 2] = v.z;
                w[4 * c4 + 3] = v.w;
            }
            // x-sums: even offsets pair points (0,1), (2,3) on aligned register pairs and
            // add into the y accumulators; odd offsets pair (1,2), points 0 and 3 scalar
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
            const float2 c0 = C::ISO ? make_float2(taylor_centre3<M>(), taylor_centre3<M>()) : p->c02;
            const float2 s0 = __fadd2_rn(__fadd2_rn(ya[r][0], yb[r][0]), make_float2(x0, xm.x));
            const float2 s1 = __fadd2_rn(__fadd2_rn(ya[r][1], yb[r][1]), make_float2(xm.y, x3));
            acc[r][0] = __ffma2_rn(c0, lo2(ctr[r]), s0);
            acc[r][1] = __ffma2_rn(c0, hi2(ctr[r]), s1);
        }
    }

    __device__ __forceinline__ float cz(int k) const { return C::ISO ? taylor<C::M>(k) : p->cz[k]; }

    // One plane iteration: plane i = za - M + it arrives.  DP: form the partial P(i)
    // (i in [za, za + nout)); DF: finish output plane j = i - M (j in [za, za + nout)).
    // A value of 2 takes the decision at run time from the iteration (one body for every
    // phase: the reverse step, whose larger epilogue gains less from specialised bodies
    // than it loses to their code size, measured on GB300).  Returns false when the loop
    // must stop.
    template <int DP_, int DF_>
    __device__ __forceinline__ bool plane(int it)
    {
        constexpr int M = C::M, RY = C::RY;
        const bool DP = DP_ == 2 ? (it >= M && it < nout + M) : DP_ != 0;
        const bool DF = DF_ == 2 ? it >= 2 * M : DF_ != 0;
        // every thread passes this barrier in every iteration, so an abort raised by any
        // thread in iteration it is seen by all of them here, in iteration it + 1
        __syncthreads();
        if (*(volatile int *)abort_flag) return false;
        if (tid == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            if (it + C::P < niter) issue_halo(it + C::P);
            const int op = it - 2 * M + C::PP;
            if (op >= 0 && op < nout) issue_pw(op);
            if (MODE == kModeAdj && C::GS) {   // g of the next output plane into L2
                const int og = it - 2 * M + 1;
                if (og >= 0 && og < nout) tma_prefetch4(me, bx * C::TX, by * C::TY, za + og, shot);
            }
        }
        if (MODE == kModeAdj && C::GS) {
            // this thread's g values of output plane j (if any) into the staging buffer,
            // whose previous contents this thread has read (in program order) already;
            // rows outside the grid copy nothing and read as zero
            const int og = it - 2 * M;
            if (og >= 0) {
                const int64_t zoff = (int64_t)(za + og) * plane_f;
#pragma unroll
                for (int r = 0; r < RY; ++r) {
                    const float *src = rowok[r] ? gp + zoff + (int64_t)r * p->px : gp;
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                                 ::"r"(smem_u32(gbuf + (ty * RY + r) * C::TX + tx * 4)), "l"(src),
                                 "r"(rowok[r] ? 16 : 0)
                                 : "memory");
                }
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        const int i = za - M + it;
        const uint32_t slot = (uint32_t)(i & (M - 1)) * 8u;   // same slot for i and i - M
        const bool hok = wait_warp(bar_h + hst, (uint32_t)hph);
        const float *hk = (const float *)(halo + hst * C::HALO_STRIDE);
        hph ^= hst + 1 == C::SH;
        hst = hst + 1 == C::SH ? 0 : hst + 1;
        if (!hok) {
            atomicExch(abort_flag, 1);
            return true;
        }
        float4 ctr[RY];
        float2 pacc[RY][2];
        if (DP) {
            lap_xy(hk, pacc, ctr);
        } else {
#pragma unroll
            for (int r = 0; r < RY; ++r) ctr[r] = *(const float4 *)(hk + (ty * RY + r + M) * C::SX + tx * 4 + M);
        }
        if (!DP && !DF) {   // warm-up: the plane only enters the raw ring
            tmem_st8(traw + slot, ctr[0], ctr[1]);
            return true;
        } else {
            // the previous iteration's TMEM stores must have landed before these loads
            tmem_wait_st();
            // planes i-1 .. i-4 and the partial P(j) (the slot P(i) will take), then, at
            // radius 8, planes i-5 .. i-8 (i - M = j)
            constexpr uint32_t RM = C::RING - 1;
            Slot8 q1, q2, q3, q4, pj;
            tmem_ld5x8(traw + ((slot - 8u) & RM), traw + ((slot - 16u) & RM),
                       traw + ((slot - 24u) & RM), traw + ((slot - 32u) & RM), tpart + slot, q1,
                       q2, q3, q4, pj);
            float2 lacc[RY][2];
            // plane i - m enters P(i) with c_m and L(j) (j = i - M) with c_{M-m}
            auto add = [&](const Slot8 &q, int m) {
                if (DP) {
                    fma4(pacc[0][0], pacc[0][1], cz(m), q.a);
                    fma4(pacc[1][0], pacc[1][1], cz(m), q.b);
                }
                if (DF) {
                    if (m < M) {
                        fma4(lacc[0][0], lacc[0][1], cz(M - m), q.a);
                        fma4(lacc[1][0], lacc[1][1], cz(M - m), q.b);
                    }
                }
            };
            if (DF) {
                // L(j) starts from P(j) and the newest plane's term c_M u(i)
                lacc[0][0] = lo2(pj.a);
                lacc[0][1] = hi2(pj.a);
                lacc[1][0] = lo2(pj.b);
                lacc[1][1] = hi2(pj.b);
                fma4(lacc[0][0], lacc[0][1], cz(M), ctr[0]);
                fma4(lacc[1][0], lacc[1][1], cz(M), ctr[1]);
            }
            add(q1, 1);
            add(q2, 2);
            add(q3, 3);
            add(q4, 4);
            if constexpr (M == 8) {
                tmem_ld4x8(traw + ((slot - 40u) & RM), traw + ((slot - 48u) & RM),
                           traw + ((slot - 56u) & RM), traw + slot, q1, q2, q3, q4);
                add(q1, 5);
                add(q2, 6);
                add(q3, 7);
                add(q4, 8);
            }
            const Slot8 uj = q4;
            // the raw slot of plane i - M = j and the partial slot of P(j) are read: refill
            tmem_st8(traw + slot, ctr[0], ctr[1]);
            if (DP)
                tmem_st8(tpart + slot, make_float4(pacc[0][0].x, pacc[0][0].y, pacc[0][1].x, pacc[0][1].y),
                         make_float4(pacc[1][0].x, pacc[1][0].y, pacc[1][1].x, pacc[1][1].y));
            if (DF) return finish(it, lacc, uj);
            return true;
        }
    }

    // The update and the epilogue of output plane j = za + it - 2M from L(j) (unscaled
    // in the isotropic instantiation) and u(j).
    __device__ __forceinline__ bool finish(int it, float2 (&lacc)[C::RY][2], const Slot8 &uj)
    {
        constexpr int M = C::M, TX = C::TX, RY = C::RY;
        const int o = it - 2 * M, j = za + o;
        const int64_t zoff = (int64_t)j * plane_f;
        const bool pok = wait_warp(bar_p + pst, (uint32_t)pph);
        const int sp = pst;
        pph ^= pst + 1 == C::SP;
        pst = pst + 1 == C::SP ? 0 : pst + 1;
        if (!pok) {
            atomicExch(abort_flag, 1);
            return true;
        }
        const float *ta = (const float *)(pw + sp * C::PW_STRIDE);
        const float *tb = ta + TX * C::TY;
        if (MODE == kModeAdj && C::GS) asm volatile("cp.async.wait_group 0;" ::: "memory");
        const float sz = szs[4 * sp + (j & 3)];
        // the rows' epilogue.  Forward modes run the source and receiver checks only in the
        // planes that hold the source node or the receivers (one uniform test per plane;
        // 552^3: forward 0.561 -> 0.535 ms, forward + store 0.617 -> 0.599 ms); the
        // reverse step keeps them in every plane (hoisted, it needs 128 registers and ran
        // 0.715 -> 0.731 ms)
        auto rows = [&](auto spec_c) {
            constexpr bool SPEC = decltype(spec_c)::value;
#pragma unroll
            for (int r = 0; r < RY; ++r) {
                const float4 cz4 = r == 0 ? uj.a : uj.b;
                float2 l0 = lacc[r][0], l1 = lacc[r][1];
                if (C::ISO) {
                    const float2 ih = make_float2(p->inv_h2, p->inv_h2);
                    l0 = __fmul2_rn(l0, ih);
                    l1 = __fmul2_rn(l1, ih);
                }
                const int toff = (ty * RY + r) * TX + tx * 4;
                const int64_t off = zoff + (int64_t)r * p->px;
                const float4 A = *(const float4 *)(ta + toff);   // prev
                const float4 B = *(const float4 *)(tb + toff);   // W
                // (2c + W lap - (1 - s) prev [+ dt^2 w at the source]) / (1 + s), evaluated as
                // prev + (2 (c - prev) + W lap [+ dt^2 w]) / (1 + s)
                const float2 m1 = make_float2(-1.0f, -1.0f), two = make_float2(2.0f, 2.0f);
                const float2 dc0 = __ffma2_rn(lo2(A), m1, lo2(cz4));
                const float2 dc1 = __ffma2_rn(hi2(A), m1, hi2(cz4));
                float2 t0 = __ffma2_rn(lo2(B), l0, __fmul2_rn(two, dc0));
                float2 t1 = __ffma2_rn(hi2(B), l1, __fmul2_rn(two, dc1));
                const bool at_src = SPEC && j == src_j && r == src_r;
                if (MODE != kModeAdj && at_src) {
                    if (src_e == 0) t0.x += srcv;
                    else if (src_e == 1) t0.y += srcv;
                    else if (src_e == 2) t1.x += srcv;
                    else t1.y += srcv;
                }
                const float syz = syr[r] + sz;
                const float2 d0 = __fadd2_rn(make_float2(sx1[0], sx1[1]), make_float2(syz, syz));
                const float2 d1 = __fadd2_rn(make_float2(sx1[2], sx1[3]), make_float2(syz, syz));
                float2 o0 = __ffma2_rn(t0, make_float2(rcp_fast(d0.x), rcp_fast(d0.y)), lo2(A));
                float2 o1 = __ffma2_rn(t1, make_float2(rcp_fast(d1.x), rcp_fast(d1.y)), hi2(A));
                if (SPEC && p->rec_map && j == p->rec_z && rowok[r]) {
                    float ov[4] = {o0.x, o0.y, o1.x, o1.y};
                    s3d::rec_epilogue<MODE>(*p, shot, y0 + r, x0, nrow, ov);
                    o0 = make_float2(ov[0], ov[1]);
                    o1 = make_float2(ov[2], ov[3]);
                }
                if (MODE != kModeAdj && domax) {
                    mxa = absmax_nan(mxa, o0.x);
                    mxa = absmax_nan(mxa, o0.y);
                    mxa = absmax_nan(mxa, o1.x);
                    mxa = absmax_nan(mxa, o1.y);
                    mxd = absmax_nan(mxd, o0.x - cz4.x);
                    mxd = absmax_nan(mxd, o0.y - cz4.y);
                    mxd = absmax_nan(mxd, o1.x - cz4.z);
                    mxd = absmax_nan(mxd, o1.y - cz4.w);
                }
                if (rowok[r]) *(float4 *)(outp + off) = make_float4(o0.x, o0.y, o1.x, o1.y);
                if (MODE == kModeStepStore && rowok[r]) {
                    // checkpoint of the input pair (c = u^n, prev = u^{n-1}) in the encode
                    // kernel's format: FP32 pair, or 16-bit a = c s_a and d = (c - prev) s_d
                    if (p->st_dtype == 0) {
                        *(float4 *)(codef + off) = cz4;
                        if (p->st_comps == 2) *(float4 *)(codef + off + p->field) = A;
                    } else {
                        *(uint2 *)(codep + off) = pack_code4(cz4, p->st_dtype, sts[0]);
                        if (p->st_comps == 2)
                            *(uint2 *)(codep + off + p->field) =
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
                    const float4 G = *(const float4 *)((C::GS ? gbuf : te) + toff);
                    float2 g0 = __ffma2_rn(lo2(Ua), l0, lo2(G));
                    float2 g1 = __ffma2_rn(hi2(Ua), l1, hi2(G));
                    if (at_src) src_image(g0, g1, cz4, B, src_e, srcv);
                    if (rowok[r]) *(float4 *)(gp + off) = make_float4(g0.x, g0.y, g1.x, g1.y);
                }
            }
        };
        if (MODE == kModeAdj || j == src_z || (p->rec_map && j == p->rec_z))
            rows(BoolC<true>{});
        else
            rows(BoolC<false>{});
        return true;
    }
};

template <class C, int MODE>
__device__ __forceinline__ void run_segment(Ctx<C, MODE> &c, int col, int z0, int z1, int tiles_x,
                                            int tiles)
{
    constexpr int M = C::M, RY = C::RY;
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
#pragma unroll
    for (int r = 0; r < RY; ++r) c.syr[r] = (c.y0 + r < p.ny) ? p.sig_y[c.y0 + r] : 0.0f;
    {
        const bool xin = c.x0 < p.nx;
#pragma unroll
        for (int r = 0; r < RY; ++r) c.rowok[r] = xin && c.y0 + r < p.ny;
        const int64_t rowbase = (int64_t)c.y0 * p.px + c.x0;
        c.plane_f = p.plane;
        c.outp = p.out + (int64_t)c.shot * p.field + rowbase;
        if (MODE == kModeAdj) c.gp = p.g + (int64_t)c.shot * p.field + rowbase;
        if (MODE == kModeStepStore) {
            c.codep = (unsigned short *)p.st_code + (int64_t)c.shot * p.st_cstride + rowbase;
            c.codef = (float *)p.st_code + (int64_t)c.shot * p.st_cstride + rowbase;
        }
        c.domax = MODE != kModeAdj && p.maxbits != nullptr;
    }
    c.src_j = -1;
    c.src_z = -1;
    c.src_r = c.src_e = 0;
    c.srcv = 0.0f;
    c.nrow = (p.n_dev ? *p.n_dev : 0) + p.n;
    if (p.src_off) {
        const int64_t s = p.src_off[c.shot];
        const int sz = (int)(s / p.plane), rem = (int)(s - (int64_t)sz * p.plane);
        const int sy = rem / p.px, sx = rem - sy * p.px;
        c.src_z = sz;
        if (sy >= c.y0 && sy < c.y0 + RY && sx >= c.x0 && sx < c.x0 + 4) {
            c.src_j = sz;
            c.src_r = sy - c.y0;
            c.src_e = sx - c.x0;
            c.srcv = p.dt2 * p.wavelet[(int64_t)c.shot * p.nt + (p.n_dev ? *p.n_dev : 0) + p.n];
        }
    }
    if (c.tid == 0 && MODE == kModeAdj)
        *(float *)c.ainv = p.aux_scale ? 1.0f / p.aux_scale[2 * c.shot] : 1.0f;
    if (c.tid == 0 && MODE == kModeStepStore) {
        ((float *)c.sts)[0] = p.st_scale[2 * c.shot];
        ((float *)c.sts)[1] = p.st_scale[2 * c.shot + 1];
    }
    __syncthreads();
    if (c.tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        for (int it = 0; it < C::P && it < c.niter; ++it) c.issue_halo(it);
    }
    // phases: warm-up (planes only enter the raw ring), partials only, partials and
    // outputs (the steady state), outputs only; with nout < M a gap of warm-up planes
    // separates the partials from the outputs
    if (MODE == kModeAdj) {
        for (int it = 0; it < c.niter; ++it)
            if (!c.template plane<2, 2>(it)) break;
    } else {
        const int e1 = 2 * M < c.nout + M ? 2 * M : c.nout + M;
        int it = 0;
        bool go = true;
        for (; go && it < M; ++it) go = c.template plane<0, 0>(it);
        for (; go && it < e1; ++it) go = c.template plane<1, 0>(it);
        for (; go && it < 2 * M; ++it) go = c.template plane<0, 0>(it);
        for (; go && it < c.nout + M; ++it) go = c.template plane<1, 1>(it);
        for (; go && it < c.niter; ++it) go = c.template plane<0, 1>(it);
    }
    if (MODE != kModeAdj && p.maxbits) {
        const unsigned a = __reduce_max_sync(0xffffffffu, __float_as_uint(c.mxa) & 0x7fffffffu);
        const unsigned d = __reduce_max_sync(0xffffffffu, __float_as_uint(c.mxd) & 0x7fffffffu);
        if ((c.tid & 31) == 0) {
            if (a) atomicMax(p.maxbits + 2 * c.shot, a);
            if (d) atomicMax(p.maxbits + 2 * c.shot + 1, d);
        }
        c.mxa = c.mxd = 0.0f;
    }
}

// Persistent launch with the schedule of k_step3d.cuh (whole-column rounds, then the
// leftover columns cut along z), two CTAs per SM.
template <int M, int P, int PP, int F, int MODE>
__global__ void __launch_bounds__((F & kHalf) ? 128 : 256, (F & kHalf) ? 4 : 2)
k_step3d_tm(const __grid_constant__ Step3dParams p, const __grid_constant__ CUtensorMap map_c,
            const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
            const __grid_constant__ CUtensorMap map_d, const __grid_constant__ CUtensorMap map_e)
{
    using C = Cfg<M, P, PP, F, MODE == kModeAdj ? ((F & kGAsync) ? 3 : 4) : 2>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // aligned by pointer arithmetic on the shared array (a round trip through an integer
    // would hide the address space, and every shared-memory read would become generic)
    unsigned char *smem = smem_raw + ((1024u - (s3d::smem_u32(smem_raw) & 1023u)) & 1023u);

    Ctx<C, MODE> c;
    c.p = &p;
    c.mc = &map_c;
    c.ma = &map_a;
    c.mb = &map_b;
    c.md = &map_d;
    c.me = &map_e;
    c.halo = smem;
    c.pw = smem + C::SH * C::HALO_STRIDE;
    c.gbuf = (float *)(c.pw + C::SP * C::PW_STRIDE);
    unsigned char *misc = (unsigned char *)c.gbuf + C::GS * C::TILE_BYTES;
    c.bar_h = (uint64_t *)misc;                      // SH + SP <= 8 barriers: bytes 0..63
    c.bar_p = c.bar_h + C::SH;
    c.abort_flag = (int *)(misc + 64);
    c.ainv = (const float *)(misc + 68);
    c.sts = (const float *)(misc + 72);               // two floats
    uint32_t *tbase = (uint32_t *)(misc + 80);
    c.szs = (float *)(misc + 128);                   // 4 floats per pointwise stage
    static_assert(C::SH + C::SP <= 8 && 4 * C::SP * 4 <= 128, "misc block layout");
    c.tid = threadIdx.x;
    c.tx = c.tid % C::NTX;
    c.ty = c.tid / C::NTX;
    c.hst = c.hph = c.pst = c.pph = c.hfill = c.pfill = 0;
    c.h_issued = c.p_issued = 0;
    c.mxa = c.mxd = 0.0f;

    const int warp = c.tid >> 5;
    if (warp == 0) tmem_alloc(tbase, C::TCOLS);
    if (c.tid == 0) {
        for (int i = 0; i < C::SH; ++i) mbar_init(c.bar_h + i, 1);
        for (int i = 0; i < C::SP; ++i) mbar_init(c.bar_p + i, 1);
        *c.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    {
        const uint32_t t = *(volatile uint32_t *)tbase;
        const uint32_t lane = (uint32_t)(32 * (warp & 3)) << 16;
        c.traw = t + lane + (uint32_t)(2 * C::RING * (warp >> 2));
        c.tpart = c.traw + C::RING;
    }

    const int tiles_x = (p.nx + C::TX - 1) / C::TX;
    const int tiles = tiles_x * ((p.ny + C::TY - 1) / C::TY);
    s3d::walk_schedule(p, tiles * p.nshots, c.abort_flag,
                       [&](int col, int z0, int z1) { run_segment(c, col, z0, z1, tiles_x, tiles); });
    if (MODE == kModeAdj && C::GS) asm volatile("cp.async.wait_all;" ::: "memory");
    // every TMEM access of the CTA is complete before warp 0 releases the columns
    tmem_wait_st();
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (warp == 0) tmem_dealloc(*(volatile uint32_t *)tbase, C::TCOLS);
    if (*(volatile int *)c.abort_flag && c.tid == 0) {
        atomicOr(p.err, 2u);
        for (int q = c.h_issued - C::SH > 0 ? c.h_issued - C::SH : 0; q < c.h_issued; ++q)
            (void)mbar_wait(c.bar_h + q % C::SH, (q / C::SH) & 1);
        for (int q = c.p_issued - C::SP > 0 ? c.p_issued - C::SP : 0; q < c.p_issued; ++q)
            (void)mbar_wait(c.bar_p + q % C::SP, (q / C::SP) & 1);
    }
}

template <int M, int F>
Step3dKernelInfo kernel_info(int mode, bool tile_g, bool half)
{
    Step3dKernelInfo k;
    if ((mode == kModeStep || mode == kModeStepStore) && half) {
        // 64 x 16 tiles, four CTAs of 4 warps per SM (the radius-8 forward modes)
        using C = Cfg<M, 2, 2, F | kHalf, 2>;
        k.fn = mode == kModeStep ? (Step3dKernel)k_step3d_tm<M, 2, 2, F | kHalf, kModeStep>
                                 : (Step3dKernel)k_step3d_tm<M, 2, 2, F | kHalf, kModeStepStore>;
        k.threads = C::NT;
        k.smem = C::SMEM;
        k.tmem_cols = (int)C::TCOLS;
    } else if (mode == kModeStep || mode == kModeStepStore) {
        using C = Cfg<M, 2, 2, F, 2>;
        k.fn = mode == kModeStep ? (Step3dKernel)k_step3d_tm<M, 2, 2, F, kModeStep>
                                 : (Step3dKernel)k_step3d_tm<M, 2, 2, F, kModeStepStore>;
        k.threads = C::NT;
        k.smem = C::SMEM;
        k.tmem_cols = (int)C::TCOLS;
    } else if (tile_g) {
        // g as a fourth TMA pointwise tile: rings of three halo and two pointwise stages
        using C = Cfg<M, 2, 1, F, 4>;
        k.fn = (Step3dKernel)k_step3d_tm<M, 2, 1, F, kModeAdj>;
        k.threads = C::NT;
        k.smem = C::SMEM;
        k.tmem_cols = (int)C::TCOLS;
    } else {
        // g staged by cp.async: rings of two halo and three pointwise stages
        using C = Cfg<M, 1, 2, F | kGAsync, 3>;
        k.fn = (Step3dKernel)k_step3d_tm<M, 1, 2, F | kGAsync, kModeAdj>;
        k.threads = C::NT;
        k.smem = C::SMEM;
        k.tmem_cols = (int)C::TCOLS;
    }
    return k;
}

}  // namespace s3tm
}  // namespace fwi
