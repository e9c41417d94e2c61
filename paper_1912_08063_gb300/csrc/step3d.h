// Parameters and launchers of the TMA-staged 3-D step kernel (k_step3d.cu) and its
// host-side tensor-map helpers (tmap.cpp).  Internal to libfwi.
#pragma once

#include <cuda.h>
#include <cstdint>
#include <cuda_runtime.h>

#include "fwi_internal.h"

namespace fwi {

constexpr int kModeStep = 0;   // out = damped leapfrog update, written over prev
constexpr int kModeStepStore = 2;   // kModeStep that also writes a checkpoint of its input
                                    // pair (st_code); a separate instantiation, so the plain
                                    // step's code is unchanged
constexpr int kModeAdj = 1;    // the same update (no source) and g += aux * (L c), with the
                               // source-point term g -= dt^2 w[n] c / W

struct Step3dParams {
    int M;
    int nx, ny, nz, px;           // computed extents and row pitch (floats)
    int64_t plane, field;         // floats per z-plane and per shot
    int nshots;
    int rounds, round_ctas;       // whole-unit rounds and the CTAs each round uses
    int rem_ctas;                 // CTAs sharing the leftover units along z
    int zparts, zfirst;           // a unit is z-part h of a tile column: planes
                                  // [h zfirst, (h + 1) zfirst), the last part up to nz;
                                  // units are numbered part-major
    int rem_first, rem_ppu;       // leftover units go to CTAs rem_first ..
                                  // rem_first + rem_ctas - 1: cut into rem_ppu aligned
                                  // pieces each (rem_ppu > 0), or as one run cut into
                                  // equal pieces that may cross units (rem_ppu = 0)
    float cx[kMaxM + 1], cy[kMaxM + 1], cz[kMaxM + 1], c0;
    float2 cy2[kMaxM + 1], cz2[kMaxM + 1], c02;   // the same weights as packed pairs
    int iso;                      // hx = hy = hz: the isotropic instantiation may run
    float inv_h2;                 // 1 / h^2 of an isotropic grid
    const float *sig_x, *sig_y, *sig_z;
    float *out;                   // the new state, over prev (in place)
    float *g;                     // kModeAdj: gradient accumulator
    const int64_t *src_off;       // may be null (kModeStep: injection; kModeAdj: g term)
    const float *wavelet;
    int nt, n;
    const int *n_dev;             // nullable: the step index is *n_dev + n
    float dt2;
    unsigned *err;                // status word: bit 1 (value 2) = a bounded wait gave up
    int aux_fmt;                  // kModeAdj: aux tile of FP32 (0) or BF16 (1) / FP16 (2)
                                  // checkpoint codes
    const float *aux_scale;       // kModeAdj with codes: per shot at [2 s] (u = code / scale)
    void *st_code;                // kModeStep, nullable: checkpoint of the input pair (c, prev)
    const float *st_scale;        //   written from the epilogue (see StepParams)
    int st_dtype, st_comps;
    int64_t st_cstride;
    unsigned *maxbits;            // kModeStep, nullable: per shot, raise [2s] to the bits of
                                  // max|out| and [2s+1] to max|out - c| (the checkpoint
                                  // codec's scales of the new state pair)
    // receivers handled in the epilogue (rec_map nullable): every receiver is the node
    // (rec_z, y, x) with rec_map[shot][y][x] = its index (-1 elsewhere); forward modes
    // write rec_tr[shot][n][r] = out, the reverse mode adds
    // inj_scale[shot][r] * inj_q[shot][inj_n][r] to out (the same two roundings as the
    // separate injection kernel)
    const int *rec_map;
    int rec_z, nrec;
    float *rec_tr;
    const float *inj_q, *inj_scale;
    int inj_n;
};

// Kernel configurations of the 3-D step: tile height, points per thread along y,
// prefetch depth, planes between shifts of the register z-queue, and option bits
// (1: packed x-sums, 2: undamped fast path).  step3d_variant() picks the configuration
// used for radius M.
// Tile height, rows per thread, prefetch depth, queue shift interval, and the option bits
// (Cfg::F) of the plain forward step (opt) and of the store and reverse modes (opt_rev);
// tm = 1 selects the kernel whose z-stream lives in tensor memory (k_step3d_tm.cuh:
// 64 x 32 tiles, two CTAs per SM; ty is then 32 and the other fields do not apply);
// tile_g = 1 makes its reverse step read g as a TMA pointwise tile instead of staging it
// with per-thread asynchronous copies.
struct Step3dVariant {
    int ty, ry, pf, u, opt, opt_rev;
    int tm;
    int tile_g = 0;
    int half = 0;   // tensor-memory forward modes: 64 x 16 tiles, 4 warps, four CTAs per SM
};
// The tensor-memory reverse step takes g as a TMA tile when a launch has at least this
// many CTAs per 64 x 32 tile column, so that its columns are cut along z into as many
// short parts or pieces (23 to 72 planes on the 232^3 to 360^3 grids measured, 3-6 %
// faster there), and stages g per thread otherwise (424^3 and up, 4-15 % faster).
constexpr int kTileGParts = 5;
Step3dVariant step3d_variant(int M, int mode);
int step3d_smem_bytes(int M);
int step3d_threads(int M);
// Resident CTAs of the 3-D step kernel of `mode` on the current device (SMs x CTAs per
// SM), for the instantiation a launch on an isotropic (iso) or anisotropic grid uses;
// -e when a CUDA call of the query failed with error e.
int step3d_resident_ctas(int M, int mode, bool iso);

// map_c: 4-D [shot][z][y][x] map of the streamed field with the halo box;
// map_a, map_b, map_d, map_e: maps of the pointwise fields prev, W, aux, g with the
// 64 x TY tile box (map_d and map_e are read in kModeAdj only).  W's map has a shot
// extent of 1.
cudaError_t launch_step3d_tma(const Step3dParams &p, int mode, int ctas,
                              const CUtensorMap &map_c, const CUtensorMap &map_a,
                              const CUtensorMap &map_b, const CUtensorMap &map_d,
                              const CUtensorMap &map_e, cudaStream_t s);

// Per-radius pieces behind the dispatch (k_step3d_m4.cu, k_step3d_m8.cu).
typedef void (*Step3dKernel)(const Step3dParams, const CUtensorMap, const CUtensorMap,
                             const CUtensorMap, const CUtensorMap, const CUtensorMap);
struct Step3dKernelInfo {
    Step3dKernel fn;
    int threads, smem;
    int tmem_cols = 0;   // tensor-memory columns each CTA allocates
};
// iso: the grid is isotropic, so an instantiation with compile-time stencil weights
// (scaled by 1 / h^2 once per point) may be returned.
Step3dKernelInfo step3d_kernel_m4(const Step3dVariant &v, int mode, bool iso = false);
Step3dKernelInfo step3d_kernel_m8(const Step3dVariant &v, int mode, bool iso = false);
// The tensor-memory kernels (k_step3d_tm8.cu, k_step3d_tm4.cu).
Step3dKernelInfo step3d_kernel_tm8(int mode, bool iso, bool tile_g, bool half);
Step3dKernelInfo step3d_kernel_tm4(int mode, bool iso, bool tile_g, bool half);

// Encodes a 4-D tensor map over shots of a field laid out as in Geom (elements of
// `elem_bytes` = 4 or 2, shots `shot_stride` elements apart), with box (bx, by, 1, 1) and
// zero fill outside [0, nx) x [0, ny) x [0, nz) x [0, nshots).
int encode_field_map(CUtensorMap *map, const void *base, const Geom &g, int nshots, int bx,
                     int by, int elem_bytes, int64_t shot_stride);

// Segment idx (0, 1, ...) of CTA k in the persistent schedule of p over `columns` tile
// columns: tile column *col, output planes [*z0, *z1).  Returns false past its last
// segment.  The kernels walk it (k = blockIdx.x) and the planner evaluates it, so both
// read the same schedule.
__host__ __device__ inline bool schedule_segment(const Step3dParams &p, int columns, int k, int idx,
                                                 int *col, int *z0, int *z1)
{
    const int S = p.zparts;
    if (k < p.round_ctas) {
        if (idx < p.rounds) {
            const int u = idx * p.round_ctas + k;
            const int h = u / columns;
            *col = u - h * columns;
            *z0 = h * p.zfirst;
            *z1 = h == S - 1 ? p.nz : *z0 + p.zfirst;
            return true;
        }
        idx -= p.rounds;
    }
    const int first = p.rounds * p.round_ctas;   // first leftover unit
    const int rem = columns * S - first;
    const int kk = k - p.rem_first;
    if (rem <= 0 || kk < 0 || kk >= p.rem_ctas) return false;
    const int zb = (S - 1) * p.zfirst;            // the leftover units lie in the last part
    const int len_u = p.nz - zb;
    if (p.rem_ppu > 0) {                          // aligned pieces, one per CTA
        if (idx > 0) return false;
        const int u = first + kk / p.rem_ppu, piece = kk % p.rem_ppu;
        const int plen = (len_u + p.rem_ppu - 1) / p.rem_ppu;
        *col = u % columns;
        *z0 = zb + piece * plen;
        *z1 = *z0 + plen < p.nz ? *z0 + plen : p.nz;
        return *z0 < *z1;
    }
    const int64_t total = (int64_t)rem * len_u;
    const int64_t len = (total + p.rem_ctas - 1) / p.rem_ctas;
    const int64_t s0 = (int64_t)kk * len;
    const int64_t s1 = s0 + len < total ? s0 + len : total;
    const int64_t start = idx == 0 ? s0 : (s0 / len_u + idx) * len_u;
    if (start >= s1) return false;
    const int64_t end = (start / len_u + 1) * len_u < s1 ? (start / len_u + 1) * len_u : s1;
    const int u = first + (int)(start / len_u);
    *col = u % columns;
    *z0 = zb + (int)(start % len_u);
    *z1 = *z0 + (int)(end - start);
    return true;
}

// 3-D map [shot][z][x] of a 2-D field (elements of elem_bytes = 4 or 2, shots
// `shot_stride` elements apart) with box (bx, 1, 1) and zero fill outside the grid.
int encode_field_map2d(CUtensorMap *map, const void *base, const Geom &g, int nshots, int bx,
                       int elem_bytes, int64_t shot_stride);

// The TMA-staged 2-D step (k_step2d_tma.cu).  maps: the streamed field with boxes of 256
// and of M columns, prev, W (one shot), and for the reverse step aux and g (each with a
// 256-column box); the launcher picks the z-chunks.
cudaError_t launch_step2d_tma(const StepParams &p, int nshots, bool imaging, const CUtensorMap *maps,
                              cudaStream_t s);

// Persistent schedule of one launch over `columns` tile columns of nz planes on
// `resident` CTAs: rounds of whole units, then the leftover units cut along z into
// pieces of at least 4M planes (each piece streams 2M warm-up planes).  A unit is a whole
// column, or, with `in_step` and fewer columns than CTAs, one of S = ceil(resident /
// columns) z-parts of a column that begin at the same z in every column: the CTAs of a
// round then stream z in step part by part, so a tile's halo planes are still in L2 when
// its neighbours read them (a field larger than L2 needs this).  With z-parts the planner
// compares equal parts (leftovers cut over all CTAs, as one run or in pieces aligned to
// the leftover units) with longer first parts whose leftover last parts go, in aligned
// pieces, to the CTAs that ran a last part, and keeps the one whose busiest CTA streams
// the fewest planes (warm-up planes included).  Fills the schedule fields of p and
// returns the grid size.
int plan_persistent(Step3dParams &p, int columns, int resident, bool in_step = false);

}  // namespace fwi
