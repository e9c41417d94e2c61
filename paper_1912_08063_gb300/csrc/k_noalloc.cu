// fwi_misfit_noalloc: the L2 misfit reduction with no device allocation.
//
// fwi_misfit allocates its per-block partial sums with stream-ordered allocation on
// every call.  Some callers cannot allow that: a host framework that has reserved all of
// the device's memory for its own pool up front, or a latency-critical loop in which an
// allocation call (and the synchronisation it may bring) is not acceptable.  This entry
// point keeps the partials in a fixed array in the library's device globals instead,
// so each call allocates nothing.
//
// The array is a file-scope __device__ variable: every device that loads the library
// holds it (32 KB) until the process exits.  Host code cannot pass the variable's name
// to a kernel (on the host it is only a stand-in, not a device address), so the first
// call on each device looks up the array's device address with cudaGetSymbolAddress,
// with that device current, and caches it per (device, context); that first call should
// therefore come before any stream capture.  A cudaDeviceReset creates a new context on
// its next use, in which the module and its array are loaded again at another address:
// the first call in the new context looks the address up again.  Every call shares the
// one array and overwrites the partials it uses (no clearing is needed: each partial is
// written before it is read), so calls that overlap on the GPU — on two streams of the
// same device — race and must be ordered by the caller.
#include <cudaTypedefs.h>

#include <mutex>
#include <string>

#include "fwi.h"
#include "fwi_internal.h"

namespace fwi {
int report_error(int code, const std::string &msg);
}

namespace {

constexpr int kThreads = 256;
constexpr int64_t kChunk = 1 << 16;        // samples summed by one block
constexpr int kMaxPartials = 4096;         // partial sums the array holds (32 KB)
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_misfit_partials[kMaxPartials];

std::mutex g_mutex;
double *g_partials_addr[kMaxDevices] = {};
CUcontext g_partials_ctx[kMaxDevices] = {};

// The current driver context (through the runtime's driver entry point, so the library
// needs no libcuda link); null when it cannot be queried.
CUcontext current_context()
{
    static PFN_cuCtxGetCurrent_v4000 get = nullptr;
    if (!get) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !f) {
            cudaGetLastError();
            return nullptr;
        }
        get = (PFN_cuCtxGetCurrent_v4000)f;
    }
    CUcontext c = nullptr;
    return get(&c) == CUDA_SUCCESS ? c : nullptr;
}

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
    return t;
}

// Block b sums samples [b * kChunk, min(n, (b + 1) * kChunk)): thread t adds
// b * kChunk + t + k * kThreads in increasing k, then a fixed tree; the order depends on
// n only, so the result is reproducible.
__global__ void k_partials(const float *__restrict__ d, const float *__restrict__ dobs, int64_t n,
                           double *__restrict__ part)
{
    const int64_t lo = blockIdx.x * kChunk;
    const int64_t hi = lo + kChunk < n ? lo + kChunk : n;
    double acc = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kThreads) {
        const float r = d[i] - dobs[i];
        acc += (double)r * (double)r;
    }
    const double t = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void k_total(const double *__restrict__ part, int nb, double *__restrict__ out)
{
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += kThreads) acc += part[i];
    const double t = block_sum(acc);
    if (threadIdx.x == 0) out[0] = t;
}

// Device address of the partials array on the current device (looked up once per device
// and context).
int partials_address(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return fwi::report_error(FWI_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return fwi::report_error(FWI_ERR_ARG, "device ordinal beyond the supported 64");
    // cudaGetSymbolAddress below makes the device's primary context current if none is,
    // so the context is read after it when the cache is empty
    std::lock_guard<std::mutex> lock(g_mutex);
    const CUcontext ctx = current_context();
    if (!g_partials_addr[dev] || !ctx || ctx != g_partials_ctx[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_misfit_partials);
        if (e != cudaSuccess || !p)
            return fwi::report_error(FWI_ERR_CUDA, std::string("cudaGetSymbolAddress: ") +
                                                       cudaGetErrorString(e));
        g_partials_addr[dev] = (double *)p;
        g_partials_ctx[dev] = ctx ? ctx : current_context();
    }
    *out = g_partials_addr[dev];
    return FWI_OK;
}

}  // namespace

extern "C" int fwi_misfit_noalloc(const float *d_mod, const float *d_obs, int64_t n,
                                  double *misfit_dev, cudaStream_t stream)
{
    if (!d_mod || !d_obs || !misfit_dev || n < 0)
        return fwi::report_error(FWI_ERR_ARG, "fwi_misfit_noalloc: null pointer or n < 0");
    if (n > kChunk * kMaxPartials)
        return fwi::report_error(
            FWI_ERR_ARG, "fwi_misfit_noalloc: n = " + std::to_string(n) +
                             " exceeds the maximum of " + std::to_string(kChunk * kMaxPartials) +
                             " samples (4096 partial sums of 65536 samples); use fwi_misfit");
    double *part = nullptr;
    const int rc = partials_address(&part);
    if (rc != FWI_OK) return rc;
    const int nb = (int)((n + kChunk - 1) / kChunk);
    // each launch is checked on its own, so the total never runs after a failed partials
    // launch (an error already pending from earlier, unrelated work is reported here too:
    // the runtime keeps one last-error slot per thread)
    if (nb > 0) {
        k_partials<<<nb, kThreads, 0, stream>>>(d_mod, d_obs, n, part);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess)
            return fwi::report_error(FWI_ERR_CUDA, std::string("fwi_misfit_noalloc (partials): ") +
                                                       cudaGetErrorString(e));
    }
    k_total<<<1, kThreads, 0, stream>>>(part, nb, misfit_dev);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fwi::report_error(FWI_ERR_CUDA, std::string("fwi_misfit_noalloc (total): ") +
                                                   cudaGetErrorString(e));
    return FWI_OK;
}
