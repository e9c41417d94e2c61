// Dispatch of the TMA-staged 3-D step kernel (template in k_step3d.cuh; the radius-4 and
// radius-8 instantiations live in k_step3d_m4.cu and k_step3d_m8.cu so they compile in
// parallel).
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include <algorithm>

#include "step3d.h"

namespace fwi {

// Configuration per radius and mode; FWI_STEP3D_VARIANT=<ty>,<ry>,<pf>,<u>,<opt>[,<opt_rev>]
// overrides the register-queue kernel's configuration for tuning runs (only the
// instantiated combinations are accepted), and FWI_STEP3D_TMEM=0/1 turns the
// tensor-memory kernel off/on in every mode, and FWI_STEP3D_TILE_G=0/1 fixes the form of
// its reverse step (g staged per thread / g as a TMA tile; unset: by the launch's CTAs
// per tile column, kTileGParts).  By default, as measured on GB300: the
// tensor-memory kernel in every mode at radius 8, and at radius 4 in the forward modes
// (forward 0.090 -> 0.087 ms, forward + store 0.108 -> 0.085 ms at 296^3) but not in the
// reverse mode (0.1165 against 0.1194 ms).  The register-queue kernel at radius 8 shifts
// its queue every 2 planes and takes the packed x-sums in all modes (measured fastest
// against U = 3 and scalar x-sums).
Step3dVariant step3d_variant(int M, int mode)
{
    Step3dVariant v = M == 8 ? Step3dVariant{32, 2, 2, 2, 1, 1, 1} : Step3dVariant{16, 2, 3, 2, 0, 0, 0};
    if (M == 4) v.tm = mode != kModeAdj;
    if (const char *e = std::getenv("FWI_STEP3D_TMEM")) v.tm = std::atoi(e) != 0;
    if (const char *e = std::getenv("FWI_STEP3D_VARIANT")) {
        int ty, ry, pf, un, opt, optr;
        const int n = std::sscanf(e, "%d,%d,%d,%d,%d,%d", &ty, &ry, &pf, &un, &opt, &optr);
        if (n == 5 || n == 6) {
            Step3dVariant w{ty, ry, pf, un, opt, n == 6 ? optr : opt, 0};
            bool ok = true;
            for (int md = 0; md < 3; ++md)
                ok = ok && (M == 8 ? step3d_kernel_m8(w, md) : step3d_kernel_m4(w, md)).fn;
            if (ok) v = w;
        }
    }
    if (v.tm) {
        // radius-8 forward modes on 64 x 16 tiles, four CTAs of 4 warps per SM (measured
        // at 552^3 against two CTAs of 8 warps: forward 0.522 -> 0.500 ms, forward + store
        // 0.577 -> 0.545 ms; at 424^3 0.282 -> 0.245 and 0.306 -> 0.266 ms); not the
        // reverse step, which fits only one halo and one pointwise stage then (552^3:
        // 0.724 -> 0.851 ms), nor radius 4 (552^3 forward 0.481 -> 0.515 ms, forward +
        // store 0.579 -> 0.617 ms);
        // FWI_STEP3D_HALF=0/1 overrides for the forward modes
        v.half = M == 8 && mode != kModeAdj;
        if (const char *e = std::getenv("FWI_STEP3D_HALF")) v.half = mode != kModeAdj && std::atoi(e) != 0;
        v.ty = v.half ? 16 : 32;
    }
    return v;
}

static Step3dKernelInfo kernel_info(int M, int mode, bool iso = false, bool tile_g = false)
{
    Step3dVariant v = step3d_variant(M, mode);
    v.tile_g = tile_g;
    if (M == 8) return step3d_kernel_m8(v, mode, iso);
    if (M == 4) return step3d_kernel_m4(v, mode, iso);
    return Step3dKernelInfo{nullptr, 0, 0};
}

int step3d_smem_bytes(int M) { return kernel_info(M, kModeStep).smem; }
int step3d_threads(int M) { return kernel_info(M, kModeStep).threads; }

// Resident CTAs per SM need the kernel's largest shared-memory carveout: with the
// driver's default preference a 101 KB reverse-step CTA at radius 4 may get a carveout
// that holds only one of them, and the persistent grid, sized for two, would then run in
// two waves.
static cudaError_t prepare_kernel(const Step3dKernelInfo &k)
{
    cudaError_t e = cudaFuncSetAttribute((const void *)k.fn,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, k.smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute((const void *)k.fn,
                                cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared);
}

static int resident_ctas(const Step3dKernelInfo &k)
{
    if (!k.fn) return -(int)cudaErrorInvalidDeviceFunction;
    cudaError_t e = prepare_kernel(k);
    int dev = 0, sms = 0, per = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess && k.tmem_cols > 0) {
        // kernels that allocate tensor memory: the occupancy query counts one CTA per SM
        // for them (measured), while their registers, shared memory and columns admit
        // more; count from those resources
        cudaFuncAttributes a{};
        int regs = 0, shm = 0, rsv = 0, thr = 0;
        e = cudaFuncGetAttributes(&a, (const void *)k.fn);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&regs, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&shm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&thr, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
        if (e == cudaSuccess) {
            const int warps = (k.threads + 31) / 32;
            const int regs_warp = (a.numRegs + 7) / 8 * 8 * 32;   // per-warp granule of 256
            per = 512 / k.tmem_cols;
            if (regs_warp > 0) per = std::min(per, regs / (regs_warp * warps));
            per = std::min(per, shm / (k.smem + (int)a.sharedSizeBytes + rsv));
            per = std::min(per, thr / k.threads);
        }
    } else if (e == cudaSuccess) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, (const void *)k.fn, k.threads, k.smem);
    }
    if (e != cudaSuccess || per < 1 || sms < 1) {
        cudaGetLastError();
        return -(int)(e != cudaSuccess ? e : cudaErrorInvalidConfiguration);
    }
    return sms * per;
}

// The reverse step's two forms (g staged per thread or as a TMA tile) are planned with
// one count: the smaller of theirs.
int step3d_resident_ctas(int M, int mode, bool iso)
{
    const int a = resident_ctas(kernel_info(M, mode, iso));
    if (mode != kModeAdj || a < 0) return a;
    const int b = resident_ctas(kernel_info(M, mode, iso, true));
    return b < 0 ? b : std::min(a, b);
}

cudaError_t launch_step3d_tma(const Step3dParams &p, int mode, int ctas,
                              const CUtensorMap &mc, const CUtensorMap &ma,
                              const CUtensorMap &mb, const CUtensorMap &md,
                              const CUtensorMap &me, cudaStream_t s)
{
    const int ty = step3d_variant(p.M, mode).ty;
    const int64_t columns = (int64_t)((p.nx + 63) / 64) * ((p.ny + ty - 1) / ty) * p.nshots;
    bool tile_g = (int64_t)ctas > (int64_t)(kTileGParts - 1) * columns;   // ctas/columns >= 5
    if (const char *e = std::getenv("FWI_STEP3D_TILE_G")) tile_g = std::atoi(e) != 0;
    const Step3dKernelInfo k = kernel_info(p.M, mode, p.iso != 0, mode == kModeAdj && tile_g);
    if (!k.fn) return cudaErrorInvalidValue;
    const cudaError_t e = prepare_kernel(k);
    if (e != cudaSuccess) return e;
    if (ctas < 1) return cudaErrorInvalidValue;
    k.fn<<<ctas, k.threads, k.smem, s>>>(p, mc, ma, mb, md, me);
    return cudaGetLastError();
}

}  // namespace fwi
