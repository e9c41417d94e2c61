// Host helpers of the TMA-staged 3-D step: tensor-map encoding (through the driver entry
// point, so the library needs no libcuda link) and the persistent schedule.
#include <cudaTypedefs.h>

#include "step3d.h"

namespace fwi {

int encode_field_map(CUtensorMap *map, const void *base, const Geom &g, int nshots, int bx,
                     int by, int elem_bytes, int64_t shot_stride)
{
    if (elem_bytes != 4 && elem_bytes != 2) return -1;
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
    const cuuint64_t eb = (cuuint64_t)elem_bytes;
    const cuuint64_t strides[3] = {(cuuint64_t)g.px * eb, (cuuint64_t)g.plane * eb,
                                   (cuuint64_t)shot_stride * eb};
    const cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    // 16-bit codes are moved as raw 16-bit words (zero fill = +0 in either format)
    const CUtensorMapDataType dt =
        elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    CUresult r = encode(map, dt, 4, const_cast<void *>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -1;
}

int plan_persistent(Step3dParams &p, int columns, int resident, bool in_step)
{
    if (resident < 1) resident = 1;
    int S = 1;
    if (in_step && columns > 0 && columns < resident) {
        S = (resident + columns - 1) / columns;
        // parts no shorter than 4M planes
        while (S > 1 && p.nz / S < 4 * p.M) --S;
        // the walk needs every leftover unit in the last part, which S = ceil(resident /
        // columns) guarantees; a thinner split keeps whole columns
        if ((long long)S * columns < resident) S = 1;
    }
    p.zparts = S;
    const int last = p.nz - (int)((long long)(S - 1) * p.nz / S);   // planes of the last part
    const long long units = (long long)columns * S;
    p.round_ctas = resident;
    p.rounds = (int)(units / resident);
    // the leftover units all lie in the last part: (S - 1) columns' worth of units fit in
    // fewer than `resident` slots when S = ceil(resident / columns)
    const long long rem_planes = (units - (long long)p.rounds * resident) * (S > 1 ? last : p.nz);
    long long pieces = rem_planes / (4LL * p.M);
    if (pieces < 1) pieces = 1;
    if (pieces > resident) pieces = resident;
    p.rem_ctas = rem_planes > 0 ? (int)pieces : 0;
    return p.rounds > 0 ? resident : (p.rem_ctas > 0 ? p.rem_ctas : 1);
}

}  // namespace fwi
