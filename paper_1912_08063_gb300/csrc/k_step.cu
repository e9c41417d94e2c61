// K1 (forward step) and K2 (adjoint step + zero-lag imaging) of the damped leapfrog,
// Eq. 3 of Huot et al. (Sec. 3) with the sponge reading: one launch advances every shot
// of a batch by one time step.
//
// Design (CUDA cores: the stencil is not a dense contraction):
//   * a CTA owns a TX x TY tile of the (x, y) plane and a chunk of z-planes and streams
//     through them along z (the slowest axis);
//   * the z-neighbours of each point live in a per-thread register queue of 2M+1
//     values, fed by one coalesced load per plane (each plane read once from HBM);
//   * the x/y-neighbours come from the current plane's tile plus an M-wide halo staged
//     in shared memory (halo reads are mostly L2 hits: neighbouring CTAs read the same
//     plane at about the same time);
//   * prev and W are read once and the new state is written once over prev:
//     16 bytes per point per step (28 with imaging: + u_img, g read and g write);
//   * the sponge factor comes from three per-axis tables (no per-point array) and the
//     source is added by the thread that owns its node.
// The adjoint reuses the same update: with mu = W nu the transposed step is the forward
// operator (2 + W L) applied to mu, because L is symmetric and W diagonal, so the
// reverse sweep needs no W halo.  Imaging then accumulates mu^{m+1} (L u^m).
#include "fwi_internal.h"

namespace fwi {

namespace {

__device__ __forceinline__ float ldz(const float *__restrict__ f, int z, int nz,
                                     int64_t plane, int64_t xy, bool inside)
{
    return (inside && z >= 0 && z < nz) ? __ldg(f + (int64_t)z * plane + xy) : 0.0f;
}

template <int M, int TX, int TY, bool IMG>
__global__ void __launch_bounds__(TX *TY) k_step3d(const StepParams p)
{
    constexpr int SX = TX + 2 * M, SY = TY + 2 * M, Q = 2 * M + 1;
    __shared__ float tile[SY][SX];
    __shared__ float tileu[IMG ? SY : 1][IMG ? SX : 1];

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int shot = blockIdx.z / p.nzchunks, zc = blockIdx.z - shot * p.nzchunks;
    const int nz = p.g.nz, ny = p.g.ny, nx = p.g.nx;
    const int z0 = zc * p.zchunk, z1 = min(nz, z0 + p.zchunk);
    const int x = x0 + tx, y = y0 + ty;
    const bool inside = (x < nx) && (y < ny);
    const int64_t plane = p.g.plane, px = p.g.px;
    const int64_t sb = (int64_t)shot * p.g.field;
    const float *__restrict__ cur = p.cur + sb;
    float *__restrict__ prev = p.prev + sb;
    const float *__restrict__ uim = IMG ? p.u_img + sb : nullptr;
    const int64_t xy = (int64_t)y * px + x;

    float q[Q];
    float qu[IMG ? Q : 1];
#pragma unroll
    for (int i = 0; i < Q - 1; ++i) {
        q[i] = ldz(cur, z0 - M + i, nz, plane, xy, inside);
        if (IMG) qu[i] = ldz(uim, z0 - M + i, nz, plane, xy, inside);
    }
    const float sxy = inside ? (p.sig_x[x] + p.sig_y[y]) : 0.0f;
    const int64_t src = (!IMG && p.src_off) ? p.src_off[shot] : -1;
    const float srcv = (src >= 0) ? p.dt2 * p.wavelet[(int64_t)shot * p.nt + p.n] : 0.0f;

    for (int z = z0; z < z1; ++z) {
        q[Q - 1] = ldz(cur, z + M, nz, plane, xy, inside);
        if (IMG) qu[Q - 1] = ldz(uim, z + M, nz, plane, xy, inside);
        __syncthreads();
        const int64_t zoff = (int64_t)z * plane;
        for (int i = tid; i < SY * SX; i += TX * TY) {
            const int sy = i / SX, sx = i - sy * SX;
            const int gy = y0 + sy - M, gx = x0 + sx - M;
            const bool ok = gy >= 0 && gy < ny && gx >= 0 && gx < nx;
            const int64_t off = zoff + (int64_t)gy * px + gx;
            tile[sy][sx] = ok ? __ldg(cur + off) : 0.0f;
            if (IMG) tileu[sy][sx] = ok ? __ldg(uim + off) : 0.0f;
        }
        __syncthreads();
        if (inside) {
            const float c = q[M];
            float lz = 0.f, ly = 0.f, lx = 0.f;
#pragma unroll
            for (int k = 1; k <= M; ++k) {
                lz = fmaf(p.c.cz[k], q[M + k] + q[M - k], lz);
                ly = fmaf(p.c.cy[k], tile[ty + M + k][tx + M] + tile[ty + M - k][tx + M], ly);
                lx = fmaf(p.c.cx[k], tile[ty + M][tx + M + k] + tile[ty + M][tx + M - k], lx);
            }
            const float lap = fmaf(p.c.c0, c, lz + ly + lx);
            const int64_t idx = zoff + xy;
            const float s = sxy + p.sig_z[z];
            float rhs = fmaf(__ldg(p.W + idx), lap, 2.0f * c) - (1.0f - s) * prev[idx];
            if (idx == src) rhs += srcv;
            prev[idx] = (s == 0.0f) ? rhs : rhs / (1.0f + s);
            if (IMG) {
                float uz = 0.f, uy = 0.f, ux = 0.f;
#pragma unroll
                for (int k = 1; k <= M; ++k) {
                    uz = fmaf(p.c.cz[k], qu[M + k] + qu[M - k], uz);
                    uy = fmaf(p.c.cy[k], tileu[ty + M + k][tx + M] + tileu[ty + M - k][tx + M], uy);
                    ux = fmaf(p.c.cx[k], tileu[ty + M][tx + M + k] + tileu[ty + M][tx + M - k], ux);
                }
                const float lu = fmaf(p.c.c0, qu[M], uz + uy + ux);
                p.gacc[sb + idx] = fmaf(c, lu, p.gacc[sb + idx]);
            }
        }
#pragma unroll
        for (int i = 0; i < Q - 1; ++i) {
            q[i] = q[i + 1];
            if (IMG) qu[i] = qu[i + 1];
        }
    }
}

template <int M, int TX, bool IMG>
__global__ void __launch_bounds__(TX) k_step2d(const StepParams p)
{
    constexpr int SX = TX + 2 * M, Q = 2 * M + 1;
    __shared__ float row[SX];
    __shared__ float rowu[IMG ? SX : 1];

    const int tx = threadIdx.x;
    const int x0 = blockIdx.x * TX;
    const int shot = blockIdx.z / p.nzchunks, zc = blockIdx.z - shot * p.nzchunks;
    const int nz = p.g.nz, nx = p.g.nx;
    const int z0 = zc * p.zchunk, z1 = min(nz, z0 + p.zchunk);
    const int x = x0 + tx;
    const bool inside = x < nx;
    const int64_t plane = p.g.plane;
    const int64_t sb = (int64_t)shot * p.g.field;
    const float *__restrict__ cur = p.cur + sb;
    float *__restrict__ prev = p.prev + sb;
    const float *__restrict__ uim = IMG ? p.u_img + sb : nullptr;

    float q[Q];
    float qu[IMG ? Q : 1];
#pragma unroll
    for (int i = 0; i < Q - 1; ++i) {
        q[i] = ldz(cur, z0 - M + i, nz, plane, x, inside);
        if (IMG) qu[i] = ldz(uim, z0 - M + i, nz, plane, x, inside);
    }
    const float sx = inside ? p.sig_x[x] : 0.0f;
    const int64_t src = (!IMG && p.src_off) ? p.src_off[shot] : -1;
    const float srcv = (src >= 0) ? p.dt2 * p.wavelet[(int64_t)shot * p.nt + p.n] : 0.0f;

    for (int z = z0; z < z1; ++z) {
        q[Q - 1] = ldz(cur, z + M, nz, plane, x, inside);
        if (IMG) qu[Q - 1] = ldz(uim, z + M, nz, plane, x, inside);
        __syncthreads();
        const int64_t zoff = (int64_t)z * plane;
        for (int i = tx; i < SX; i += TX) {
            const int gx = x0 + i - M;
            const bool ok = gx >= 0 && gx < nx;
            row[i] = ok ? __ldg(cur + zoff + gx) : 0.0f;
            if (IMG) rowu[i] = ok ? __ldg(uim + zoff + gx) : 0.0f;
        }
        __syncthreads();
        if (inside) {
            const float c = q[M];
            float lz = 0.f, lx = 0.f;
#pragma unroll
            for (int k = 1; k <= M; ++k) {
                lz = fmaf(p.c.cz[k], q[M + k] + q[M - k], lz);
                lx = fmaf(p.c.cx[k], row[tx + M + k] + row[tx + M - k], lx);
            }
            const float lap = fmaf(p.c.c0, c, lz + lx);
            const int64_t idx = zoff + x;
            const float s = sx + p.sig_z[z];
            float rhs = fmaf(__ldg(p.W + idx), lap, 2.0f * c) - (1.0f - s) * prev[idx];
            if (idx == src) rhs += srcv;
            prev[idx] = (s == 0.0f) ? rhs : rhs / (1.0f + s);
            if (IMG) {
                float uz = 0.f, ux = 0.f;
#pragma unroll
                for (int k = 1; k <= M; ++k) {
                    uz = fmaf(p.c.cz[k], qu[M + k] + qu[M - k], uz);
                    ux = fmaf(p.c.cx[k], rowu[tx + M + k] + rowu[tx + M - k], ux);
                }
                const float lu = fmaf(p.c.c0, qu[M], uz + ux);
                p.gacc[sb + idx] = fmaf(c, lu, p.gacc[sb + idx]);
            }
        }
#pragma unroll
        for (int i = 0; i < Q - 1; ++i) {
            q[i] = q[i + 1];
            if (IMG) qu[i] = qu[i + 1];
        }
    }
}

constexpr int kTX3 = 32, kTY3 = 8, kTX2 = 128;

template <int M, bool IMG>
cudaError_t launch_m(const StepParams &p0, int nshots, cudaStream_t s)
{
    StepParams p = p0;
    const int sms = 152;
    if (p.g.ndim == 3) {
        const int bx = (p.g.nx + kTX3 - 1) / kTX3, by = (p.g.ny + kTY3 - 1) / kTY3;
        int64_t tiles = (int64_t)bx * by * nshots;
        int want = (int)((4LL * sms + tiles - 1) / tiles);
        int maxchunks = p.g.nz / (4 * M) > 0 ? p.g.nz / (4 * M) : 1;
        int nch = want < 1 ? 1 : (want > maxchunks ? maxchunks : want);
        p.zchunk = (p.g.nz + nch - 1) / nch;
        p.nzchunks = (p.g.nz + p.zchunk - 1) / p.zchunk;
        dim3 grid(bx, by, p.nzchunks * nshots), block(kTX3, kTY3);
        k_step3d<M, kTX3, kTY3, IMG><<<grid, block, 0, s>>>(p);
    } else {
        const int bx = (p.g.nx + kTX2 - 1) / kTX2;
        int64_t tiles = (int64_t)bx * nshots;
        int want = (int)((8LL * sms + tiles - 1) / tiles);
        int maxchunks = p.g.nz / (2 * M) > 0 ? p.g.nz / (2 * M) : 1;
        int nch = want < 1 ? 1 : (want > maxchunks ? maxchunks : want);
        p.zchunk = (p.g.nz + nch - 1) / nch;
        p.nzchunks = (p.g.nz + p.zchunk - 1) / p.zchunk;
        dim3 grid(bx, 1, p.nzchunks * nshots), block(kTX2);
        k_step2d<M, kTX2, IMG><<<grid, block, 0, s>>>(p);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_step(const StepParams &p, int nshots, bool imaging, cudaStream_t s)
{
    if (p.g.M == 4) return imaging ? launch_m<4, true>(p, nshots, s) : launch_m<4, false>(p, nshots, s);
    if (p.g.M == 8) return imaging ? launch_m<8, true>(p, nshots, s) : launch_m<8, false>(p, nshots, s);
    return cudaErrorInvalidValue;
}

}  // namespace fwi
