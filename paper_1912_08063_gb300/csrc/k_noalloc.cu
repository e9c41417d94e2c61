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
// with that device current, and caches it; that first call should therefore come before
// any stream capture.  Every call shares the one array and overwrites the partials it
// uses (no clearing is needed: each partial is written before it is read), so calls
// that overlap on the GPU — on two streams of the same device — race and must be
// ordered by the caller.
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

// Device address of the partials array on the current device (looked up once per device).
int partials_address(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return fwi::report_error(FWI_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return fwi::report_error(FWI_ERR_ARG, "device ordinal beyond the supported 64");
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_partials_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_misfit_partials);
        if (e != cudaSuccess || !p)
            return fwi::report_error(FWI_ERR_CUDA, std::string("cudaGetSymbolAddress: ") +
                                                       cudaGetErrorString(e));
        g_partials_addr[dev] = (double *)p;
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
    if (nb > 0) k_partials<<<nb, kThreads, 0, stream>>>(d_mod, d_obs, n, part);
    k_total<<<1, kThreads, 0, stream>>>(part, nb, misfit_dev);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fwi::report_error(FWI_ERR_CUDA, std::string("fwi_misfit_noalloc: ") +
                                                   cudaGetErrorString(e));
    return FWI_OK;
}
