// Host helpers of the TMA-staged 3-D step: tensor-map encoding (through the driver entry
// point, so the library needs no libcuda link) and the z-chunk planner.
#include <cudaTypedefs.h>

#include "step3d.h"

namespace fwi {

int encode_field_map(CUtensorMap *map, const void *base, const Geom &g, int nshots, int bx,
                     int by)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000,
                                             cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !f) {
            cudaGetLastError();
            return -1;
        }
        encode = (PFN_cuTensorMapEncodeTiled_v12000)f;
    }
    const cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz,
                                (cuuint64_t)nshots};
    const cuuint64_t strides[3] = {(cuuint64_t)g.px * 4, (cuuint64_t)g.plane * 4,
                                   (cuuint64_t)g.field * 4};
    const cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void *>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -1;
}

int plan_zchunks(int nz, int M, int tiles_per_shot, int nshots, int resident)
{
    if (resident < 1) resident = 1;
    double best = -1.0;
    int best_c = 1;
    for (int c = 1; c <= 64 && c <= nz; ++c) {
        const int zc = (nz + c - 1) / c;
        const int cn = (nz + zc - 1) / zc;
        const long long ctas = (long long)tiles_per_shot * nshots * cn;
        const long long waves = (ctas + resident - 1) / resident;
        const double fill = (double)ctas / ((double)waves * resident);
        // each chunk streams 2M extra planes that produce no output; they cost about
        // half an output plane (loads and queue pushes, no stencil)
        const double cost = 1.0 + 0.5 * (2.0 * M) / zc;
        const double score = fill / cost;
        if (score > best + 1e-9) {
            best = score;
            best_c = cn;
        }
    }
    return best_c;
}

}  // namespace fwi
