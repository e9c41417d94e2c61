// Off-grid sources and receivers: sampling, injection and the point terms of the
// transposed imaging sum for points given as Kaiser-windowed sinc taps (the tap tables
// are built on the host, api.cpp).  A point's taps are the nodes (z0 + a, y0 + b, x0 + c),
// a, c < 8 and b < ty (8 in 3-D, 1 in 2-D), with weight wz[a] wy[b] wx[c].  Sampling
// sums the weighted taps; every injection spreads a value over the same taps with the
// same weights, so injection is the exact transpose of sampling.  One thread handles one
// (point, a, b) row of 8 taps; rows of different points may overlap, so writes are
// atomic.
#include "code16.cuh"
#include "fwi_internal.h"

namespace fwi {

namespace {

constexpr int kThreads = 256;

struct TapRow {
    int64_t off;    // field offset of tap (a, b, 0)
    float wzy;      // wz[a] * wy[b]
    int z, y, x0;   // node coordinates of tap (a, b, 0)
};

__device__ __forceinline__ TapRow tap_row(const Geom &g, const PointTaps &p, int a, int b)
{
    TapRow t;
    t.z = p.z0 + a;
    t.y = p.y0 + b;
    t.x0 = p.x0;
    t.off = (int64_t)t.z * g.plane + (int64_t)t.y * g.px + t.x0;
    t.wzy = p.w[a] * p.w[kTaps + b];
    return t;
}

__device__ __forceinline__ int rows_per_point(const Geom &g) { return kTaps * (g.ndim == 3 ? kTaps : 1); }

// traces[s][n][r] = sum over taps of w * f (FP32)
__global__ void k_sample_pts(Geom g, const float *__restrict__ f, const PointTaps *__restrict__ pts,
                             int nshots, int nrec, int nt, int n, float *__restrict__ traces,
                             const int *__restrict__ n_dev)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nshots * nrec) return;
    if (n_dev) n += *n_dev;
    const int s = i / nrec, r = i - s * nrec;
    const PointTaps &p = pts[i];
    const float *fs = f + (int64_t)s * g.field;
    const int ty = g.ndim == 3 ? kTaps : 1;
    float acc = 0.0f;
    for (int a = 0; a < kTaps; ++a)
        for (int b = 0; b < ty; ++b) {
            const TapRow t = tap_row(g, p, a, b);
            float row = 0.0f;
#pragma unroll
            for (int c = 0; c < kTaps; ++c) row = fmaf(p.w[2 * kTaps + c], fs[t.off + c], row);
            acc = fmaf(t.wzy, row, acc);
        }
    traces[((int64_t)s * nt + n) * nrec + r] = acc;
}

// kind 0: forward source, f += dt^2 w[s][n] wt / a+                   (q = wavelets)
// kind 1: adjoint injection, f += factor (W / a+) wt q[s][n][r]        (q = residuals)
__global__ void k_inject_pts(Geom g, float *__restrict__ f, const PointTaps *__restrict__ pts,
                             int npts, int per_shot, const float *__restrict__ W,
                             const float *__restrict__ sz, const float *__restrict__ sy,
                             const float *__restrict__ sx, const float *__restrict__ q, int nt,
                             int n, float dt2, float factor, int kind, const int *__restrict__ n_dev)
{
    const int rows = rows_per_point(g);
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)npts * rows) return;
    if (n_dev) n += *n_dev;
    const int pi = (int)(i / rows), ab = (int)(i - (int64_t)pi * rows);
    const int ty = g.ndim == 3 ? kTaps : 1;
    const int a = ab / ty, b = ab - a * ty;
    const int s = pi / per_shot, r = pi - s * per_shot;
    const PointTaps &p = pts[pi];
    const float val = kind == 0 ? dt2 * q[(int64_t)s * nt + n]
                                : q[((int64_t)s * nt + n) * per_shot + r];
    const TapRow t = tap_row(g, p, a, b);
    float *fs = f + (int64_t)s * g.field;
    const float syz = sz[t.z] + (g.ndim == 3 ? sy[t.y] : 0.0f);
#pragma unroll
    for (int c = 0; c < kTaps; ++c) {
        const float ap = 1.0f + syz + sx[t.x0 + c];
        const float scale = kind == 0 ? 1.0f / ap : factor * W[t.off + c] / ap;
        atomicAdd(fs + t.off + c, val * t.wzy * p.w[2 * kTaps + c] * scale);
    }
}

// Point terms of the transposed imaging sum at reverse step m:
// kind 0 (source): g -= dt^2 w[s][m] wt mu^{m+1} / W            (x = mu^{m+1}, FP32)
// kind 1 (receiver): g += 2 wt u^m r[s][m-1][r]                  (x = u^m, FP32 or a code)
__global__ void k_image_pts(Geom g, float *__restrict__ gacc, const void *__restrict__ x,
                            int xfmt, int64_t xstride, const float *__restrict__ xscale,
                            const PointTaps *__restrict__ pts, int npts, int per_shot,
                            const float *__restrict__ W, const float *__restrict__ q, int nt,
                            int n, float dt2, int kind)
{
    const int rows = rows_per_point(g);
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)npts * rows) return;
    const int pi = (int)(i / rows), ab = (int)(i - (int64_t)pi * rows);
    const int ty = g.ndim == 3 ? kTaps : 1;
    const int a = ab / ty, b = ab - a * ty;
    const int s = pi / per_shot, r = pi - s * per_shot;
    const PointTaps &p = pts[pi];
    const float val = kind == 0 ? -dt2 * q[(int64_t)s * nt + n]
                                : 2.0f * q[((int64_t)s * nt + n) * per_shot + r];
    const TapRow t = tap_row(g, p, a, b);
    const float inv = (xfmt != 0 && xscale) ? 1.0f / xscale[2 * s] : 1.0f;
    float *gs = gacc + (int64_t)s * g.field;
#pragma unroll
    for (int c = 0; c < kTaps; ++c) {
        const int64_t o = t.off + c;
        float xv;
        if (xfmt == 0) xv = ((const float *)x)[(int64_t)s * xstride + o];
        else xv = code16_to_float(((const unsigned short *)x)[(int64_t)s * xstride + o], xfmt) * inv;
        if (kind == 0) xv = xv / W[o];
        atomicAdd(gs + o, val * t.wzy * p.w[2 * kTaps + c] * xv);
    }
}

// x[s][n] = dt^2 sum_t wt mu[t] / W[t]  (the wavelet-space adjoint read at the source
// taps: nu = mu / W, as the on-grid read-out at the single node)
__global__ void k_gather_src_pts(Geom g, const float *__restrict__ f,
                                 const PointTaps *__restrict__ pts, int nshots,
                                 const float *__restrict__ W, float dt2, int nt, int n,
                                 float *__restrict__ xout)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nshots) return;
    const PointTaps &p = pts[s];
    const float *fs = f + (int64_t)s * g.field;
    const int ty = g.ndim == 3 ? kTaps : 1;
    float acc = 0.0f;
    for (int a = 0; a < kTaps; ++a)
        for (int b = 0; b < ty; ++b) {
            const TapRow t = tap_row(g, p, a, b);
            for (int c = 0; c < kTaps; ++c)
                acc += t.wzy * p.w[2 * kTaps + c] * fs[t.off + c] / W[t.off + c];
        }
    xout[(int64_t)s * nt + n] = dt2 * acc;
}

unsigned blocks(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

}  // namespace

cudaError_t launch_sample_pts(const Geom &g, const float *f, const PointTaps *pts, int nshots,
                              int nrec, int nt, int n, float *traces, cudaStream_t s,
                              const int *n_dev)
{
    k_sample_pts<<<blocks((int64_t)nshots * nrec), kThreads, 0, s>>>(g, f, pts, nshots, nrec, nt,
                                                                     n, traces, n_dev);
    return cudaGetLastError();
}

cudaError_t launch_inject_pts(const Geom &g, float *f, const PointTaps *pts, int npts,
                              int per_shot, const float *W, const float *sig_z,
                              const float *sig_y, const float *sig_x, const float *q, int nt,
                              int n, float dt2, float factor, int kind, cudaStream_t s,
                              const int *n_dev)
{
    const int64_t rows = (int64_t)npts * kTaps * (g.ndim == 3 ? kTaps : 1);
    k_inject_pts<<<blocks(rows), kThreads, 0, s>>>(g, f, pts, npts, per_shot, W, sig_z, sig_y,
                                                   sig_x, q, nt, n, dt2, factor, kind, n_dev);
    return cudaGetLastError();
}

cudaError_t launch_image_pts(const Geom &g, float *gacc, const void *x, int xfmt,
                             int64_t xstride, const float *xscale, const PointTaps *pts,
                             int npts, int per_shot, const float *W, const float *q, int nt,
                             int n, float dt2, int kind, cudaStream_t s)
{
    const int64_t rows = (int64_t)npts * kTaps * (g.ndim == 3 ? kTaps : 1);
    k_image_pts<<<blocks(rows), kThreads, 0, s>>>(g, gacc, x, xfmt, xstride, xscale, pts, npts,
                                                  per_shot, W, q, nt, n, dt2, kind);
    return cudaGetLastError();
}

cudaError_t launch_gather_src_pts(const Geom &g, const float *f, const PointTaps *pts,
                                  int nshots, const float *W, float dt2, int nt, int n,
                                  float *x, cudaStream_t s)
{
    k_gather_src_pts<<<blocks(nshots), kThreads, 0, s>>>(g, f, pts, nshots, W, dt2, nt, n, x);
    return cudaGetLastError();
}

}  // namespace fwi
