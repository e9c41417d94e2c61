// Auxiliary kernels of the FWI hot path: model set-up (W = v^2 dt^2 on the padded grid),
// receiver sampling and adjoint injection, the FP64 misfit reduction (Eq. 1), the
// checkpoint codec (BF16/FP16 with a per-checkpoint power-of-two scale), the FP32 -> FP64
// gradient fold and the gradient finish (dW/dv and the fold of sponge cells).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fwi_internal.h"

namespace fwi {

namespace {

constexpr int kThreads = 256;

int blocks_for(int64_t n, int cap = 148 * 16)
{
    int64_t b = (n + kThreads - 1) / kThreads;
    if (b < 1) b = 1;
    return (int)(b > cap ? cap : b);
}

// ---------------------------------------------------------------- set-up

// W[c] = (v[clamp(c - nb)] dt)^2 on the computed grid, zero in the row padding.
// One CTA per computed row (z, y) at a time, threads along x (the row split is one 32-bit
// division per row, not two 64-bit ones per point).
__global__ void k_build_W(Geom g, int nb, int npz, int npy, int npx, const float *__restrict__ v,
                          double dt, float *__restrict__ W)
{
    const int nby = (g.ndim == 3) ? nb : 0;
    const int rows = g.nz * g.ny;
    for (int row = blockIdx.x; row < rows; row += gridDim.x) {
        const int z = row / g.ny, y = row - z * g.ny;
        const int pz = min(max(z - nb, 0), npz - 1), py = min(max(y - nby, 0), npy - 1);
        const float *vr = v + ((int64_t)pz * npy + py) * npx;
        float *wr = W + (int64_t)row * g.px;
        for (int x = threadIdx.x; x < g.px; x += blockDim.x) {
            float w = 0.0f;
            if (x < g.nx) {
                const double vv = vr[min(max(x - nb, 0), npx - 1)];
                w = (float)(vv * vv * dt * dt);
            }
            wr[x] = w;
        }
    }
}

// out[i] = factor * W / (1 + s)  (mode 0: adjoint receiver injection of W R^T q / a+)
// out[i] = factor / W            (mode 1: source read-out dt^2 mu / W)
__global__ void k_rec_scale(Geom g, const float *__restrict__ W, const float *__restrict__ sz,
                            const float *__restrict__ sy, const float *__restrict__ sx,
                            const int64_t *__restrict__ off, int count, float factor, int mode,
                            float *__restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int64_t o = off[i];
    const int64_t z = o / g.plane, r = o - z * g.plane;
    const int64_t y = r / g.px, x = r - y * g.px;
    const float w = W[o];
    if (mode == 0) {
        const float s = sz[z] + sy[y] + sx[x];
        out[i] = factor * w / (1.0f + s);
    } else {
        out[i] = factor / w;
    }
}

// ---------------------------------------------------------------- receivers

__global__ void k_sample(int64_t fs, const float *__restrict__ f, const int64_t *__restrict__ off,
                         int nshots, int nrec, int nt, int n, float *__restrict__ traces,
                         const int *__restrict__ n_dev)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nshots * nrec) return;
    const int s = i / nrec, r = i - s * nrec;
    if (n_dev) n += *n_dev;
    traces[((int64_t)s * nt + n) * nrec + r] = f[(int64_t)s * fs + off[i]];
}

__global__ void k_inject(int64_t fs, float *__restrict__ f, const int64_t *__restrict__ off,
                         const float *__restrict__ scale, const float *__restrict__ q,
                         int nshots, int nrec, int nt, int sample)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nshots * nrec) return;
    const int s = i / nrec, r = i - s * nrec;
    atomicAdd(f + (int64_t)s * fs + off[i], scale[i] * q[((int64_t)s * nt + sample) * nrec + r]);
}

// One thread per (shot, receiver): 2 sum_k d (d - dobs) in FP64, with the residual rounded
// to FP32 exactly as the misfit kernel rounds it (the value injected into the adjoint).
__global__ void k_rec_image(int64_t fs, const float *__restrict__ d,
                            const float *__restrict__ dobs, const int64_t *__restrict__ off,
                            int nshots, int nrec, int nt, double *__restrict__ g)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nshots * nrec) return;
    const int s = i / nrec, r = i - s * nrec;
    double acc = 0.0;
    for (int k = 0; k < nt; ++k) {
        const int64_t t = ((int64_t)s * nt + k) * nrec + r;
        const float dd = d[t];
        const float rr = dd - dobs[t];
        acc = fma(2.0 * (double)dd, (double)rr, acc);
    }
    atomicAdd(g + (int64_t)s * fs + off[i], acc);
}

// One thread per shot: g[src] -= dt^2 w[0] mu^1[src] / W[src], the m = 0 source term of
// the transposed imaging sum (the reverse sweep ends with the step that makes mu^1).
__global__ void k_src_image(int64_t fs, const float *__restrict__ mu1,
                            const int64_t *__restrict__ off, const float *__restrict__ W,
                            const float *__restrict__ wav, float dt2, int nshots, int nt,
                            double *__restrict__ g)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nshots) return;
    const int64_t o = off[s];
    const float f0 = dt2 * wav[(int64_t)s * nt];
    g[(int64_t)s * fs + o] -= (double)f0 * (double)mu1[(int64_t)s * fs + o] / (double)W[o];
}

__global__ void k_gather_src(int64_t fs, const float *__restrict__ f,
                             const int64_t *__restrict__ off, const float *__restrict__ sc,
                             int nshots, int nt, int sample, float *__restrict__ x)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nshots) return;
    x[(int64_t)s * nt + sample] = f[(int64_t)s * fs + off[s]] * sc[s];
}

// ---------------------------------------------------------------- misfit (Eq. 1)

__device__ double block_sum(double v)
{
    __shared__ double part[kThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) part[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (wid == 0) {
        t = lane < kThreads / 32 ? part[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    return t;  // valid in thread 0
}

// Fixed-order partial sums: thread t of block b adds samples b*T + t + k*(B*T), k = 0.. in
// order, then a fixed tree.  The grid size depends only on n, so the result is
// reproducible bit for bit.
__global__ void k_misfit_partial(const float *__restrict__ d, const float *__restrict__ dobs,
                                 float *__restrict__ r_out, int64_t n, double *__restrict__ part)
{
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kThreads) {
        const float r = d[i] - dobs[i];
        if (r_out) r_out[i] = r;
        acc += (double)r * (double)r;
    }
    const double t = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void k_sum_partials(const double *__restrict__ part, int nb, double *__restrict__ out,
                               unsigned *flag)
{
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += kThreads) acc += part[i];
    const double t = block_sum(acc);
    if (threadIdx.x == 0) {
        out[0] = t;
        if (flag && !isfinite(t)) atomicOr(flag, 1u);
    }
}

// ---------------------------------------------------------------- checkpoint codec

__device__ __forceinline__ unsigned absbits(float x) { return __float_as_uint(x) & 0x7fffffffu; }

// out[2s] = bits of max|a|, out[2s+1] = bits of max|a - b| (FP32 difference) per shot s;
// a NaN or infinity anywhere in a or b drives both to >= 0x7f800000.
__global__ void k_maxabs(const float *__restrict__ a, const float *__restrict__ b, int64_t n,
                         int64_t stride, unsigned *__restrict__ out)
{
    const int s = blockIdx.y;
    const float *pa = a + s * stride, *pb = b + s * stride;
    unsigned ma = 0, md = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float x = pa[i], y = pb[i];
        const unsigned bad = (absbits(x) >= 0x7f800000u || absbits(y) >= 0x7f800000u) ? 0x7fc00000u : 0u;
        ma = max(ma, max(absbits(x), bad));
        md = max(md, max(absbits(x - y), bad));
    }
    ma = __reduce_max_sync(0xffffffffu, ma);
    md = __reduce_max_sync(0xffffffffu, md);
    if ((threadIdx.x & 31) == 0) {
        if (ma) atomicMax(out + 2 * s, ma);
        if (md) atomicMax(out + 2 * s + 1, md);
    }
}

// s = 2^floor(log2(T / max)) with T = 2^texp, from the bit pattern of max (exact
// integer arithmetic); NaN for a non-finite max, 1 for an all-zero pair.
__device__ float snap_scale(unsigned mb, int dtype)
{
    if (dtype == 0 || mb == 0u) return 1.0f;
    if (mb >= 0x7f800000u) return __int_as_float(0x7fc00000);
    const int texp = (dtype == 2) ? 14 : 0;
    const unsigned e = mb >> 23, mant = mb & 0x7fffffu;
    int E;
    bool frac;
    if (e > 0) {
        E = (int)e - 127;
        frac = mant != 0u;
    } else {
        E = (31 - __clz((int)mant)) - 149;
        frac = (mant & (mant - 1u)) != 0u;
    }
    int k = texp - E - (frac ? 1 : 0);
    k = max(-126, min(127, k));
    return __int_as_float((k + 127) << 23);
}

// One thread per shot: the checkpoint scales from the max-abs bits (as k_encode derives
// them), for a store that the next forward step writes from its epilogue.
__global__ void k_snap_scales(const unsigned *__restrict__ maxbits, int nshots, int dtype,
                              float *__restrict__ scale, unsigned *flag)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nshots) return;
    scale[2 * s] = snap_scale(maxbits[2 * s], dtype);
    scale[2 * s + 1] = snap_scale(maxbits[2 * s + 1], dtype);
    if (flag && maxbits[2 * s] >= 0x7f800000u) atomicOr(flag, 1u);
}

// One value of the codec: FP32 copy, or x * scale rounded to the 16-bit format.
__device__ __forceinline__ void put_code(void *code, int64_t i, int dtype, float x, float sc)
{
    if (dtype == 0) ((float *)code)[i] = x;
    else if (dtype == 1) ((__nv_bfloat16 *)code)[i] = __float2bfloat16_rn(x * sc);
    else ((__half *)code)[i] = __float2half_rn(x * sc);
}

// inv = 1 / scale.  Scales are powers of two (2^-126 .. 2^127), so their reciprocals are
// exact and code * inv equals code / scale bit for bit.
__device__ __forceinline__ float get_code(const void *code, int64_t i, int dtype, float inv)
{
    if (dtype == 0) return ((const float *)code)[i];
    if (dtype == 1) return __bfloat162float(((const __nv_bfloat16 *)code)[i]) * inv;
    return __half2float(((const __half *)code)[i]) * inv;
}

// 16-bit formats store a = u^n and d = u^n - u^{n-1}, each with its own scale; FP32
// stores the pair unchanged (lossless).  comps = 1 stores or restores a only (a
// checkpoint that is only ever restored for an imaging step, which needs u^n alone).
// VEC processes four values per thread (n a multiple of 4, 16-byte aligned fields).
template <bool VEC>
__global__ void k_encode(const float *__restrict__ a, const float *__restrict__ b, int64_t n,
                         int64_t stride, int dtype, const unsigned *__restrict__ maxbits,
                         void *__restrict__ code, int64_t cstride, float *__restrict__ scale,
                         unsigned *flag, int comps)
{
    const int s = blockIdx.y;
    const float sa = snap_scale(maxbits[2 * s], dtype);
    const float sd = snap_scale(maxbits[2 * s + 1], dtype);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        scale[2 * s] = sa;
        scale[2 * s + 1] = sd;
        if (flag && maxbits[2 * s] >= 0x7f800000u) atomicOr(flag, 1u);
    }
    const float *pa = a + s * stride, *pb = b + s * stride;
    const int esz = dtype == 0 ? 4 : 2;
    void *ca = (char *)code + (size_t)s * cstride * esz;
    void *cd = (char *)ca + (size_t)n * esz;
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    if (VEC) {
        for (int64_t i4 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i4 < n / 4; i4 += step) {
            const float4 va = ((const float4 *)pa)[i4];
            float4 vb = make_float4(0.f, 0.f, 0.f, 0.f);
            if (comps == 2) vb = ((const float4 *)pb)[i4];
            if (dtype == 0) {
                ((float4 *)ca)[i4] = va;
                if (comps == 2) ((float4 *)cd)[i4] = vb;
                continue;
            }
            const float xa[4] = {va.x, va.y, va.z, va.w};
            const float xd[4] = {va.x - vb.x, va.y - vb.y, va.z - vb.z, va.w - vb.w};
            unsigned short ha[4], hd[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (dtype == 1) {
                    ha[e] = __bfloat16_as_ushort(__float2bfloat16_rn(xa[e] * sa));
                    hd[e] = __bfloat16_as_ushort(__float2bfloat16_rn(xd[e] * sd));
                } else {
                    ha[e] = __half_as_ushort(__float2half_rn(xa[e] * sa));
                    hd[e] = __half_as_ushort(__float2half_rn(xd[e] * sd));
                }
            }
            ((ushort4 *)ca)[i4] = make_ushort4(ha[0], ha[1], ha[2], ha[3]);
            if (comps == 2) ((ushort4 *)cd)[i4] = make_ushort4(hd[0], hd[1], hd[2], hd[3]);
        }
    } else {
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += step) {
            const float va = pa[i];
            put_code(ca, i, dtype, va, sa);
            if (comps == 2) {
                const float vb = pb[i];
                put_code(cd, i, dtype, dtype == 0 ? vb : va - vb, sd);
            }
        }
    }
}

template <bool VEC>
__global__ void k_decode(const void *__restrict__ code, int64_t cstride,
                         const float *__restrict__ scale, int64_t n, int64_t stride, int dtype,
                         float *__restrict__ a, float *__restrict__ b, int comps)
{
    const int s = blockIdx.y;
    const float sa = 1.0f / scale[2 * s], sd = 1.0f / scale[2 * s + 1];   // exact: powers of 2
    float *pa = a + s * stride, *pb = b + s * stride;
    const int esz = dtype == 0 ? 4 : 2;
    const void *ca = (const char *)code + (size_t)s * cstride * esz;
    const void *cd = (const char *)ca + (size_t)n * esz;
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    if (VEC) {
        for (int64_t i4 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i4 < n / 4; i4 += step) {
            if (dtype == 0) {
                ((float4 *)pa)[i4] = ((const float4 *)ca)[i4];
                if (comps == 2) ((float4 *)pb)[i4] = ((const float4 *)cd)[i4];
                continue;
            }
            const ushort4 ua = ((const ushort4 *)ca)[i4];
            const unsigned short ha[4] = {ua.x, ua.y, ua.z, ua.w};
            float xa[4], xb[4];
#pragma unroll
            for (int e = 0; e < 4; ++e)
                xa[e] = (dtype == 1 ? __bfloat162float(__ushort_as_bfloat16(ha[e]))
                                    : __half2float(__ushort_as_half(ha[e]))) * sa;
            ((float4 *)pa)[i4] = make_float4(xa[0], xa[1], xa[2], xa[3]);
            if (comps == 2) {
                const ushort4 ud = ((const ushort4 *)cd)[i4];
                const unsigned short hd[4] = {ud.x, ud.y, ud.z, ud.w};
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    xb[e] = xa[e] - (dtype == 1 ? __bfloat162float(__ushort_as_bfloat16(hd[e]))
                                                : __half2float(__ushort_as_half(hd[e]))) * sd;
                ((float4 *)pb)[i4] = make_float4(xb[0], xb[1], xb[2], xb[3]);
            }
        }
    } else {
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += step) {
            const float va = get_code(ca, i, dtype, sa);
            pa[i] = va;
            if (comps == 2) {
                const float v = get_code(cd, i, dtype, sd);
                pb[i] = dtype == 0 ? v : va - v;
            }
        }
    }
}

__global__ void k_nonfinite(const float *__restrict__ a, int64_t n, unsigned *flag)
{
    unsigned bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        bad |= absbits(a[i]) >= 0x7f800000u;
    bad = __reduce_or_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0 && bad) atomicOr(flag, 1u);
}

// ---------------------------------------------------------------- gradient

__global__ void k_fold(float *__restrict__ g32, double *__restrict__ g64, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        g64[i] += (double)g32[i];
        g32[i] = 0.0f;
    }
}

// grad(p) = (2 / v(p)) * sum_shots sum_{computed cells c replicated from p} g_mu(c),
// where g_mu = sum_m mu^{m+1} L u^m and mu = W nu (so dphi/dW = g_mu / W and
// dphi/dv = 2 v dt^2 dphi/dW = 2 g_mu / v).
// One CTA per physical row (pz, py) at a time, threads along x.
__global__ void k_finish(Geom g, int nb, int npz, int npy, int npx, int nshots,
                         const double *__restrict__ g64, const float *__restrict__ v,
                         float *__restrict__ grad32, double *__restrict__ grad64)
{
    const int nby = (g.ndim == 3) ? nb : 0;
    const int rows = npz * npy;
    for (int row = blockIdx.x; row < rows; row += gridDim.x) {
        const int pz = row / npy, py = row - pz * npy;
        const int z0 = pz == 0 ? 0 : pz + nb, z1 = pz == npz - 1 ? pz + 2 * nb : pz + nb;
        const int y0 = py == 0 ? 0 : py + nby, y1 = py == npy - 1 ? py + 2 * nby : py + nby;
        for (int pxx = threadIdx.x; pxx < npx; pxx += blockDim.x) {
            const int x0 = pxx == 0 ? 0 : pxx + nb, x1 = pxx == npx - 1 ? pxx + 2 * nb : pxx + nb;
            double acc = 0.0;
            for (int s = 0; s < nshots; ++s) {
                const double *gs = g64 + (int64_t)s * g.field;
                for (int cz = z0; cz <= z1; ++cz)
                    for (int cy = y0; cy <= y1; ++cy)
                        for (int cx = x0; cx <= x1; ++cx)
                            acc += gs[(int64_t)cz * g.plane + (int64_t)cy * g.px + cx];
            }
            const int64_t i = (int64_t)row * npx + pxx;
            const double out = acc * 2.0 / (double)v[i];
            if (grad32) grad32[i] = (float)out;
            if (grad64) grad64[i] = out;
        }
    }
}

}  // namespace

// ---------------------------------------------------------------- launchers

cudaError_t launch_build_W(const Geom &g, int nb, const int64_t np[3], const float *v,
                           float dt, float *W, cudaStream_t s)
{
    const int rows = g.nz * g.ny;
    k_build_W<<<rows < 152 * 16 ? rows : 152 * 16, kThreads, 0, s>>>(g, nb, (int)np[0], (int)np[1],
                                                                     (int)np[2], v, dt, W);
    return cudaGetLastError();
}

__global__ void k_tick(int *counter, int add, int set)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *counter = set ? add : *counter + add;
}

cudaError_t launch_tick(int *counter, int add, cudaStream_t s)
{
    k_tick<<<1, 32, 0, s>>>(counter, add, 0);
    return cudaGetLastError();
}

cudaError_t launch_set_counter(int *counter, int value, cudaStream_t s)
{
    k_tick<<<1, 32, 0, s>>>(counter, value, 1);
    return cudaGetLastError();
}

cudaError_t launch_sample(const Geom &g, const float *field, const int64_t *rec_off,
                          int nshots, int nrec, int nt, int n, float *traces, cudaStream_t s,
                          const int *n_dev)
{
    int cnt = nshots * nrec;
    k_sample<<<(cnt + kThreads - 1) / kThreads, kThreads, 0, s>>>(g.field, field, rec_off,
                                                                 nshots, nrec, nt, n, traces,
                                                                 n_dev);
    return cudaGetLastError();
}

cudaError_t launch_inject(const Geom &g, float *field, const int64_t *rec_off,
                          const float *scale, const float *q, int nshots, int nrec, int nt,
                          int sample, cudaStream_t s)
{
    int cnt = nshots * nrec;
    k_inject<<<(cnt + kThreads - 1) / kThreads, kThreads, 0, s>>>(g.field, field, rec_off,
                                                                 scale, q, nshots, nrec, nt,
                                                                 sample);
    return cudaGetLastError();
}

cudaError_t launch_rec_image(const Geom &g, const float *d, const float *dobs,
                             const int64_t *rec_off, int nshots, int nrec, int nt,
                             double *gacc64, cudaStream_t s)
{
    int cnt = nshots * nrec;
    if (cnt <= 0 || nt <= 0) return cudaSuccess;
    k_rec_image<<<(cnt + kThreads - 1) / kThreads, kThreads, 0, s>>>(g.field, d, dobs, rec_off,
                                                                     nshots, nrec, nt, gacc64);
    return cudaGetLastError();
}

cudaError_t launch_src_image(const Geom &g, const float *mu1, const int64_t *src_off,
                             const float *W, const float *wavelet, float dt2, int nshots,
                             int nt, double *gacc64, cudaStream_t s)
{
    if (nshots <= 0) return cudaSuccess;
    k_src_image<<<(nshots + kThreads - 1) / kThreads, kThreads, 0, s>>>(
        g.field, mu1, src_off, W, wavelet, dt2, nshots, nt, gacc64);
    return cudaGetLastError();
}

cudaError_t launch_snap_scales(const unsigned *maxbits, int nshots, int dtype, float *scale,
                               unsigned *flag, cudaStream_t s)
{
    if (nshots <= 0) return cudaSuccess;
    k_snap_scales<<<(nshots + kThreads - 1) / kThreads, kThreads, 0, s>>>(maxbits, nshots, dtype,
                                                                         scale, flag);
    return cudaGetLastError();
}

cudaError_t launch_gather_src(const Geom &g, const float *field, const int64_t *src_off,
                              const float *src_scale, int nshots, int nt, int sample,
                              float *x, cudaStream_t s)
{
    k_gather_src<<<(nshots + 63) / 64, 64, 0, s>>>(g.field, field, src_off, src_scale, nshots,
                                                   nt, sample, x);
    return cudaGetLastError();
}

cudaError_t launch_rec_scale(const Geom &g, const float *W, const float *sig_z,
                             const float *sig_y, const float *sig_x, const int64_t *off,
                             int count, float factor, int mode, float *out, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    k_rec_scale<<<(count + kThreads - 1) / kThreads, kThreads, 0, s>>>(g, W, sig_z, sig_y,
                                                                      sig_x, off, count,
                                                                      factor, mode, out);
    return cudaGetLastError();
}

int misfit_blocks(int64_t n) { return blocks_for(n, 1024); }

cudaError_t launch_misfit(const float *d, const float *dobs, float *r_out, int64_t n,
                          double *partials, int nblocks, double *result, unsigned *flag,
                          cudaStream_t s)
{
    k_misfit_partial<<<nblocks, kThreads, 0, s>>>(d, dobs, r_out, n, partials);
    k_sum_partials<<<1, kThreads, 0, s>>>(partials, nblocks, result, flag);
    return cudaGetLastError();
}

cudaError_t launch_maxabs(const float *a, const float *b, int64_t n, int64_t stride,
                          int nshots, unsigned *maxbits, cudaStream_t s)
{
    dim3 grid(blocks_for(n, 152 * 8), nshots);
    k_maxabs<<<grid, kThreads, 0, s>>>(a, b, n, stride, maxbits);
    return cudaGetLastError();
}

static bool vec_ok(int64_t n, int64_t stride, int64_t code_stride, const void *x, const void *y,
                   const void *code)
{
    auto al = [](const void *p, int k) { return ((uintptr_t)p % k) == 0; };
    return n % 4 == 0 && stride % 4 == 0 && code_stride % 4 == 0 && al(x, 16) && al(y, 16) &&
           al(code, 16);
}

cudaError_t launch_encode(const float *a, const float *b, int64_t n, int64_t stride,
                          int nshots, int dtype, const unsigned *maxbits, void *code,
                          int64_t code_stride, float *scale, unsigned *flag, int comps,
                          cudaStream_t s)
{
    if (vec_ok(n, stride, code_stride, a, b, code)) {
        dim3 grid(blocks_for(n / 4, 152 * 8), nshots);
        k_encode<true><<<grid, kThreads, 0, s>>>(a, b, n, stride, dtype, maxbits, code,
                                                 code_stride, scale, flag, comps);
    } else {
        dim3 grid(blocks_for(n, 152 * 8), nshots);
        k_encode<false><<<grid, kThreads, 0, s>>>(a, b, n, stride, dtype, maxbits, code,
                                                  code_stride, scale, flag, comps);
    }
    return cudaGetLastError();
}

cudaError_t launch_decode(const void *code, int64_t code_stride, const float *scale,
                          int64_t n, int64_t stride, int nshots, int dtype, float *a, float *b,
                          int comps, cudaStream_t s)
{
    if (vec_ok(n, stride, code_stride, a, b, code)) {
        dim3 grid(blocks_for(n / 4, 152 * 8), nshots);
        k_decode<true><<<grid, kThreads, 0, s>>>(code, code_stride, scale, n, stride, dtype, a,
                                                 b, comps);
    } else {
        dim3 grid(blocks_for(n, 152 * 8), nshots);
        k_decode<false><<<grid, kThreads, 0, s>>>(code, code_stride, scale, n, stride, dtype, a,
                                                  b, comps);
    }
    return cudaGetLastError();
}

cudaError_t launch_fold(float *g32, double *g64, int64_t n, cudaStream_t s)
{
    k_fold<<<blocks_for(n, 152 * 8), kThreads, 0, s>>>(g32, g64, n);
    return cudaGetLastError();
}

cudaError_t launch_finish(const Geom &g, int nb, const int64_t np[3], int nshots,
                          const double *g64, const float *v, float *grad32, double *grad64,
                          cudaStream_t s)
{
    const int rows = (int)(np[0] * np[1]);
    k_finish<<<rows < 152 * 16 ? rows : 152 * 16, kThreads, 0, s>>>(
        g, nb, (int)np[0], (int)np[1], (int)np[2], nshots, g64, v, grad32, grad64);
    return cudaGetLastError();
}

cudaError_t launch_nonfinite_check(const float *a, int64_t n, unsigned *flag, cudaStream_t s)
{
    k_nonfinite<<<blocks_for(n, 152 * 4), kThreads, 0, s>>>(a, n, flag);
    return cudaGetLastError();
}

}  // namespace fwi
