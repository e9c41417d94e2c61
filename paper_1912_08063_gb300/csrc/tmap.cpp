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

int encode_field_map2d(CUtensorMap *map, const void *base, const Geom &g, int nshots, int bx,
                       int elem_bytes, int64_t shot_stride)
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
    const cuuint64_t eb = (cuuint64_t)elem_bytes;
    const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.nz, (cuuint64_t)nshots};
    const cuuint64_t strides[2] = {(cuuint64_t)g.px * eb, (cuuint64_t)shot_stride * eb};
    const cuuint32_t box[3] = {(cuuint32_t)bx, 1, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType dt =
        elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    CUresult r = encode(map, dt, 3, const_cast<void *>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -1;
}

// Planes (with warm-up) the busiest CTA streams under schedule p.
static int64_t schedule_cost(const Step3dParams &p, int columns, int grid)
{
    int64_t worst = 0;
    for (int k = 0; k < grid; ++k) {
        int64_t it = 0;
        int col, z0, z1;
        for (int i = 0; schedule_segment(p, columns, k, i, &col, &z0, &z1); ++i) it += z1 - z0 + 2 * p.M;
        if (it > worst) worst = it;
    }
    return worst;
}

int plan_persistent(Step3dParams &p, int columns, int resident, bool in_step)
{
    if (resident < 1) resident = 1;
    if (columns < 1) columns = 1;
    // whole columns: rounds, then the leftover columns cut into pieces of >= 4M planes
    p.zparts = 1;
    p.zfirst = p.nz;
    p.round_ctas = resident;
    p.rounds = columns / resident;
    p.rem_first = 0;
    p.rem_ppu = 0;
    {
        const long long rem_planes = (long long)(columns - p.rounds * resident) * p.nz;
        long long pieces = rem_planes / (4LL * p.M);
        if (pieces < 1) pieces = 1;
        if (pieces > resident) pieces = resident;
        p.rem_ctas = rem_planes > 0 ? (int)pieces : 0;
    }
    int grid = p.rounds > 0 ? resident : (p.rem_ctas > 0 ? p.rem_ctas : 1);
    if (!in_step || columns >= resident) return grid;

    const int S = (resident + columns - 1) / columns;   // (S - 1) columns < resident
    if (p.nz / S < 4 * p.M) return grid;                 // parts too thin: whole columns
    Step3dParams best = p;
    int64_t best_cost = -1;
    int best_grid = grid;
    // (a) equal parts; the leftover last parts cut over all CTAs
    {
        Step3dParams q = p;
        q.zparts = S;
        q.zfirst = p.nz / S;
        q.rounds = 1;
        q.rem_first = 0;
        q.rem_ppu = 0;
        const long long rem_planes = (long long)(columns * S - resident) * (p.nz - (S - 1) * q.zfirst);
        long long pieces = rem_planes / (4LL * p.M);
        if (pieces < 1) pieces = 1;
        if (pieces > resident) pieces = resident;
        q.rem_ctas = rem_planes > 0 ? (int)pieces : 0;
        const int64_t c = schedule_cost(q, columns, resident);
        best = q;
        best_cost = c;
        best_grid = resident;
    }
    // (c) equal parts; the leftover last parts in aligned pieces over all CTAs
    {
        const int L = columns * S - resident;
        const int ppu = L > 0 ? resident / L : 0;
        if (ppu >= 1) {
            Step3dParams q = best;
            q.rem_first = 0;
            q.rem_ppu = ppu;
            q.rem_ctas = L * ppu;
            const int64_t c = schedule_cost(q, columns, resident);
            if (c < best_cost) {
                best = q;
                best_cost = c;
            }
        }
    }
    // (b) longer first parts; the L leftover last parts go in ppu aligned pieces to the
    // qn CTAs that ran a last part, with lengths that balance both kinds of CTA:
    // first part + 2M = last part + 2M + last part / ppu + 2M
    {
        const int qn = resident - (S - 1) * columns, L = columns - qn;
        const int ppu = L > 0 ? qn / L : 0;
        if (L > 0 && ppu >= 1) {
            const double ll = (double)(p.nz - 2 * p.M * (S - 1)) / ((S - 1) * (1.0 + 1.0 / ppu) + 1.0);
            Step3dParams q = p;
            q.zparts = S;
            q.zfirst = (int)((p.nz - ll) / (S - 1) + 0.5);
            const int last = p.nz - (S - 1) * q.zfirst;
            if (last >= 2 * p.M && q.zfirst >= 4 * p.M) {
                q.rounds = 1;
                q.rem_first = (S - 1) * columns;
                q.rem_ppu = ppu;
                q.rem_ctas = L * ppu;
                const int64_t c = schedule_cost(q, columns, resident);
                if (c < best_cost) {
                    best = q;
                    best_cost = c;
                }
            }
        }
    }
    const Step3dParams keep = p;
    p = keep;
    p.zparts = best.zparts;
    p.zfirst = best.zfirst;
    p.rounds = best.rounds;
    p.round_ctas = best.round_ctas;
    p.rem_first = best.rem_first;
    p.rem_ppu = best.rem_ppu;
    p.rem_ctas = best.rem_ctas;
    return best_grid;
}

}  // namespace fwi
