// fwi_selftest_wait: the failure path of the step kernels' bounded waits, exercised
// without a fault.
//
// The 3-D step kernels wait on mbarriers that TMA copies complete; if the data never
// arrive, a wait gives up after a bounded number of polls, the CTA raises bit 1 of the
// model's status word, and the host reports FWI_ERR_TIMEOUT.  This kernel reaches the
// same branch on purpose: one thread arms an mbarrier with an expected transaction count
// (the arrive the step kernels' producer makes before its copy), issues no copy, and
// waits with the step kernels' own bounded wait at a small poll limit.  The phase cannot
// complete, the wait runs out, and the status bit is raised exactly as a step kernel
// would raise it.  No copy is ever in flight, so nothing can land in shared memory after
// the CTA exits; the thread then completes the missing transaction bytes itself so the
// barrier ends in a completed phase.
#include <string>

#include "fwi.h"
#include "k_step3d.cuh"

namespace fwi {
int report_error(int code, const std::string &msg);

namespace {

__global__ void k_wait_selftest(unsigned *err, int polls)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    s3d::mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s3d::mbar_expect_tx(&bar, 16);   // the arrival happens; 16 bytes stay outstanding
    if (!s3d::mbar_wait(&bar, 0, polls)) {
        atomicOr(err, 2u);   // the step kernels' timeout bit
        asm volatile("mbarrier.complete_tx.shared::cta.b64 [%0], %1;" ::"r"(s3d::smem_u32(&bar)),
                     "r"(16)
                     : "memory");
        (void)s3d::mbar_wait(&bar, 0, polls);
    }
}

}  // namespace

cudaError_t launch_wait_selftest(unsigned *err, int polls, cudaStream_t s)
{
    k_wait_selftest<<<1, 32, 0, s>>>(err, polls);
    return cudaGetLastError();
}

}  // namespace fwi
