// 2-D time step on GB300 (sm_103a) with TMA-staged rows.
//
// A CTA of 64 threads owns a 256-column x tile of one shot and a chunk of rows; it streams
// along z.  One elected thread issues, P rows ahead, the TMA copies of each new row of
// the streamed field (three boxes: the M halo columns left of the tile, the tile's 256
// columns, the M halo columns right of it, each in its own 128-byte aligned region; out
// of the grid the TMA unit fills zeros, the Dirichlet condition) into a ring of
// M + 1 + P stages, and the copies of the output row's pointwise operands (prev and W;
// the reverse step adds u^m, read as FP32 or in place as a 16-bit checkpoint code, and
// g) into a ring of PP + 1 stages; mbarriers with transaction counts signal arrival and
// every wait is bounded.  Each thread keeps the 2M + 1 rows of its 4 columns in a
// register queue (z-neighbours) and reads the x-window of the output row from the
// resident halo stage (it arrived M rows earlier and the ring keeps it).  The arithmetic
// of a point is lap4/update4 (step2d_math.cuh), as in every 2-D step kernel, so results
// equal the register-streaming kernel's bit for bit.  What changes is where the latency
// goes: the loads of a row are issued P rows before it is used and land in shared
// memory, so they neither hold registers nor stall the arithmetic that consumes them.
// DRAM traffic per point and step: 16 bytes forward (12 + 4 / shots for a batch sharing
// W), 26 or 28 reverse.
#include <cuda.h>

#include "code16.cuh"
#include "fwi_internal.h"
#include "k_step3d.cuh"
#include "step2d_math.cuh"

namespace fwi {
namespace {

using s3d::mbar_expect_tx;
using s3d::mbar_init;
using s3d::mbar_wait;
using s3d::smem_u32;

// One box of a 3-D map [shot][z][x] (coordinates x, z, shot) into shared memory.
__device__ __forceinline__ void tma_load3(void *dst, const CUtensorMap *map, int x, int z, int shot,
                                          uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(z), "r"(shot), "r"(smem_u32(bar))
        : "memory");
}
using s2d::hi2;
using s2d::lap4;
using s2d::lo2;
using s2d::update4;

constexpr int kT = 64;          // threads per CTA
constexpr int kTX = 4 * kT;     // columns per tile

template <int M, bool IMG>
struct Cfg2 {
    static constexpr int P = 4, PP = 3;            // rows prefetched: halo, pointwise
    static constexpr int SH = M + 1 + P, SP = PP + 1;
    static constexpr int SIDE = 128;               // bytes of a halo side region
    static constexpr int HSTAGE = 2 * SIDE + kTX * 4;   // left | body | right
    static constexpr int NPW = IMG ? 4 : 2;        // pointwise rows per stage
    static constexpr int PSTAGE = NPW * kTX * 4;
    static constexpr int SMEM = SH * HSTAGE + SP * PSTAGE + 256 + 128;
};

// Streams rows [za - M, za + nout + M) of tile bx, shot `shot`; outputs rows [za, za + nout).
template <int M, bool IMG, bool STORE>
__global__ void __launch_bounds__(kT) k_step2d_tma(const __grid_constant__ StepParams p,
                                                   const __grid_constant__ CUtensorMap mc_body,
                                                   const __grid_constant__ CUtensorMap mc_side,
                                                   const __grid_constant__ CUtensorMap m_prev,
                                                   const __grid_constant__ CUtensorMap m_W,
                                                   const __grid_constant__ CUtensorMap m_aux,
                                                   const __grid_constant__ CUtensorMap m_g)
{
    using C = Cfg2<M, IMG>;
    constexpr int Q = 2 * M + 1, W4 = M / 4;
    extern __shared__ __align__(128) unsigned char sm_raw[];
    unsigned char *sm = sm_raw + ((128u - (smem_u32(sm_raw) & 127u)) & 127u);
    unsigned char *halo = sm;
    unsigned char *pw = sm + C::SH * C::HSTAGE;
    uint64_t *bar_h = (uint64_t *)(pw + C::SP * C::PSTAGE);
    uint64_t *bar_p = bar_h + C::SH;
    int *abort_flag = (int *)(bar_p + C::SP);
    static_assert((C::SH + C::SP) * 8 + 4 <= 256, "barrier block");

    const int tid = threadIdx.x;
    const int shot = blockIdx.z / p.nzchunks, zc = blockIdx.z - shot * p.nzchunks;
    const int nz = p.g.nz, nx = p.g.nx;
    const int za = zc * p.zchunk, zend = min(nz, za + p.zchunk);
    const int nout = zend - za, niter = nout + 2 * M;
    const int X0 = blockIdx.x * kTX;
    const int x0 = X0 + 4 * tid;
    const bool xin = x0 < nx;
    const int64_t plane = p.g.plane;
    const int64_t sb = (int64_t)shot * p.g.field;
    const int n = (p.n_dev ? *p.n_dev : 0) + p.n;
    const int afmt = p.aux_fmt;
    const float ainv = (IMG && p.aux_scale) ? 1.0f / p.aux_scale[2 * shot] : 1.0f;
    const uint32_t pw_bytes =
        IMG ? (afmt != 0 ? 3 * kTX * 4 + kTX * 2 : 4 * kTX * 4) : 2 * kTX * 4;

    if (tid == 0) {
        for (int i = 0; i < C::SH; ++i) mbar_init(bar_h + i, 1);
        for (int i = 0; i < C::SP; ++i) mbar_init(bar_p + i, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // copies: row za - M + it of the streamed field into halo stage it % SH, pointwise
    // row za + o into stage o % SP (3-D maps over [shot][z][x])
    auto issue_halo = [&](int it) {
        const int st = it % C::SH;
        uint64_t *b = bar_h + st;
        unsigned char *d = halo + st * C::HSTAGE;
        const int z = za - M + it;
        mbar_expect_tx(b, kTX * 4 + 2 * M * 4);
        tma_load3(d, &mc_side, X0 - M, z, shot, b);
        tma_load3(d + C::SIDE, &mc_body, X0, z, shot, b);
        tma_load3(d + C::SIDE + kTX * 4, &mc_side, X0 + kTX, z, shot, b);
    };
    auto issue_pw = [&](int o) {
        const int st = o % C::SP;
        uint64_t *b = bar_p + st;
        unsigned char *d = pw + st * C::PSTAGE;
        const int z = za + o;
        mbar_expect_tx(b, pw_bytes);
        tma_load3(d, &m_prev, X0, z, shot, b);
        tma_load3(d + kTX * 4, &m_W, X0, z, 0, b);
        if (IMG) {
            tma_load3(d + 2 * kTX * 4, &m_aux, X0, z, shot, b);
            tma_load3(d + 3 * kTX * 4, &m_g, X0, z, shot, b);
        }
    };
    int h_issued = 0, p_issued = 0;
    if (tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        for (int it = 0; it < C::P && it < niter; ++it) issue_halo(it);
        for (int o = 0; o < C::PP && o < nout; ++o) issue_pw(o);
        h_issued = min(C::P, niter);
        p_issued = min(C::PP, nout);
    }

    float sx[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) sx[e] = (x0 + e < nx) ? p.sig_x[x0 + e] : 0.0f;
    int src_z = -1, src_e = 0;
    float srcv = 0.0f;
    if (p.src_off) {
        const int64_t so = p.src_off[shot];
        const int sz = (int)(so / plane), sxx = (int)(so - (int64_t)sz * plane);
        if (sxx >= x0 && sxx < x0 + 4) {
            src_z = sz;
            src_e = sxx - x0;
            srcv = p.dt2 * p.wavelet[(int64_t)shot * p.nt + n];
        }
    }
    unsigned mxa = 0u, mxd = 0u;
    float sca = 1.0f, scd = 1.0f;
    if (STORE && p.st_dtype != 0) {
        sca = p.st_scale[2 * shot];
        scd = p.st_scale[2 * shot + 1];
    }
    float *__restrict__ prev = p.prev + sb;

    float4 q[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) q[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int it = 0; it < niter; ++it) {
        __syncthreads();   // every thread is done with the stages refilled below
        if (*(volatile int *)abort_flag) break;
        if (tid == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            if (it + C::P < niter) {
                issue_halo(it + C::P);
                ++h_issued;
            }
            const int op = it - 2 * M + C::PP;
            if (op >= C::PP && op < nout) {
                issue_pw(op);
                ++p_issued;
            }
        }
        const int st = it % C::SH;
        if (!mbar_wait(bar_h + st, (it / C::SH) & 1)) {
            atomicExch(abort_flag, 1);
            continue;
        }
        // the new row enters the queue
#pragma unroll
        for (int i = 0; i < Q - 1; ++i) q[i] = q[i + 1];
        q[Q - 1] = *(const float4 *)(halo + st * C::HSTAGE + C::SIDE + 16 * tid);
        if (it < 2 * M) continue;

        const int o = it - 2 * M, z = za + o;
        const int sp = o % C::SP;
        if (!mbar_wait(bar_p + sp, (o / C::SP) & 1)) {
            atomicExch(abort_flag, 1);
            continue;
        }
        // x-window of output row z: its halo stage arrived M rows ago
        const int sj = (st + C::SH - M) % C::SH;
        const unsigned char *hj = halo + sj * C::HSTAGE;
        float w[4 + 2 * M];
#pragma unroll
        for (int g4 = 0; g4 < 2 * W4 + 1; ++g4) {
            float4 v;
            if (g4 == W4) {
                v = q[M];
            } else {
                const int c = 4 * tid + 4 * (g4 - W4);   // tile column of the group
                const unsigned char *src = c < 0 ? hj + 4 * (c + M)
                                           : c >= kTX ? hj + C::SIDE + kTX * 4 + 4 * (c - kTX)
                                                      : hj + C::SIDE + 4 * c;
                v = *(const float4 *)src;
            }
            w[4 * g4] = v.x, w[4 * g4 + 1] = v.y, w[4 * g4 + 2] = v.z, w[4 * g4 + 3] = v.w;
        }
        float2 l0, l1;
        lap4<M>(w, q, p.c, l0, l1);
        const float4 c = q[M];
        if (xin) {
            const unsigned char *ps = pw + sp * C::PSTAGE;
            const float4 pv = *(const float4 *)(ps + 16 * tid);
            const float4 Wv = *(const float4 *)(ps + kTX * 4 + 16 * tid);
            const int64_t row = (int64_t)z * plane;
            const float4 ov = update4(c, l0, l1, pv, Wv, sx, p.sig_z[z],
                                      (!IMG && z == src_z) ? src_e : -1, srcv);
            const float rhs[4] = {ov.x, ov.y, ov.z, ov.w};
            *(float4 *)(prev + row + x0) = ov;
            if (STORE) {
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
                const float4 uv = afmt == 0
                                      ? *(const float4 *)(ps + 2 * kTX * 4 + 16 * tid)
                                      : unpack_code4(*(const uint2 *)(ps + 2 * kTX * 4 + 8 * tid),
                                                     afmt, ainv);
                const float4 gv = *(const float4 *)(ps + 3 * kTX * 4 + 16 * tid);
                float2 g0 = __ffma2_rn(lo2(uv), l0, lo2(gv));
                float2 g1 = __ffma2_rn(hi2(uv), l1, hi2(gv));
                if (z == src_z) {
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
    }
    if (!IMG && p.maxbits) {
        const unsigned a = __reduce_max_sync(0xffffffffu, mxa);
        const unsigned d = __reduce_max_sync(0xffffffffu, mxd);
        if ((threadIdx.x & 31) == 0) {
            if (a) atomicMax(p.maxbits + 2 * shot, a);
            if (d) atomicMax(p.maxbits + 2 * shot + 1, d);
        }
    }
    __syncthreads();
    if (*(volatile int *)abort_flag && tid == 0) {
        // a bounded wait gave up: report, then give every copy still in flight a bounded
        // chance to land before the CTA's shared memory is released
        atomicOr(p.err, 2u);
        for (int k = max(0, h_issued - C::SH); k < h_issued; ++k)
            (void)mbar_wait(bar_h + k % C::SH, (k / C::SH) & 1);
        for (int k = max(0, p_issued - C::SP); k < p_issued; ++k)
            (void)mbar_wait(bar_p + k % C::SP, (k / C::SP) & 1);
    }
}

template <int M, bool IMG, bool STORE>
int resident_tma2()
{
    static const int r = [] {
        using C = Cfg2<M, IMG>;
        const void *fn = (const void *)k_step2d_tma<M, IMG, STORE>;
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kT, C::SMEM) != cudaSuccess || per < 1) {
            cudaGetLastError();
            per = 1;
        }
        return (sms > 0 ? sms : 152) * per;
    }();
    return r;
}

template <int M, bool IMG, bool STORE>
cudaError_t launch_tma2(const StepParams &p0, int nshots, const CUtensorMap *maps, cudaStream_t s)
{
    using C = Cfg2<M, IMG>;
    StepParams p = p0;
    const int bx = (p.g.nx + kTX - 1) / kTX;
    const int64_t ctas = (int64_t)bx * nshots;
    const int resident = resident_tma2<M, IMG, STORE>();
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
    const dim3 grid(bx, 1, p.nzchunks * nshots);
    const void *fn = (const void *)k_step2d_tma<M, IMG, STORE>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    k_step2d_tma<M, IMG, STORE><<<grid, kT, C::SMEM, s>>>(p, maps[0], maps[1], maps[2], maps[3],
                                                         maps[4], maps[5]);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_step2d_tma(const StepParams &p, int nshots, bool imaging, const CUtensorMap *maps,
                              cudaStream_t s)
{
    const bool store = !imaging && p.st_code;
    if (p.g.M == 4)
        return imaging ? launch_tma2<4, true, false>(p, nshots, maps, s)
               : store ? launch_tma2<4, false, true>(p, nshots, maps, s)
                       : launch_tma2<4, false, false>(p, nshots, maps, s);
    if (p.g.M == 8)
        return imaging ? launch_tma2<8, true, false>(p, nshots, maps, s)
               : store ? launch_tma2<8, false, true>(p, nshots, maps, s)
                       : launch_tma2<8, false, false>(p, nshots, maps, s);
    return cudaErrorInvalidValue;
}

}  // namespace fwi
