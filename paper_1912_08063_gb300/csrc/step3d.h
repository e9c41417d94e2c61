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
    int zparts;                   // a unit is z-part h, planes [h nz / zparts,
                                  // (h + 1) nz / zparts), of a tile column; units are
                                  // numbered part-major
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
};

// Kernel configurations of the 3-D step: tile height, points per thread along y,
// prefetch depth, planes between shifts of the register z-queue, and option bits
// (1: packed x-sums, 2: undamped fast path).  step3d_variant() picks the configuration
// used for radius M.
// Tile height, rows per thread, prefetch depth, queue shift interval, and the option bits
// (Cfg::F) of the plain forward step (opt) and of the store and reverse modes (opt_rev);
// tm = 1 selects the radius-8 kernel whose z-stream lives in tensor memory
// (k_step3d_tm.cuh: 64 x 32 tiles, two CTAs per SM; the other fields then do not apply).
struct Step3dVariant {
    int ty, ry, pf, u, opt, opt_rev;
    int tm;
};
Step3dVariant step3d_variant(int M);
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
// The tensor-memory radius-8 kernel (k_step3d_tm8.cu).
Step3dKernelInfo step3d_kernel_tm8(int mode, bool iso);

// Encodes a 4-D tensor map over shots of a field laid out as in Geom (elements of
// `elem_bytes` = 4 or 2, shots `shot_stride` elements apart), with box (bx, by, 1, 1) and
// zero fill outside [0, nx) x [0, ny) x [0, nz) x [0, nshots).
int encode_field_map(CUtensorMap *map, const void *base, const Geom &g, int nshots, int bx,
                     int by, int elem_bytes, int64_t shot_stride);

// Persistent schedule of one launch over `columns` tile columns of nz planes on
// `resident` CTAs: rounds of whole units, then the leftover units cut along z into
// pieces of at least 4M planes (each piece streams 2M warm-up planes).  A unit is a whole
// column, or, with `in_step` and fewer columns than CTAs, one of S = ceil(resident /
// columns) z-parts of a column that begin at the same z in every column: the CTAs of a
// round then stream z in step part by part, so a tile's halo planes are still in L2 when
// its neighbours read them (a field larger than L2 needs this).  Fills p.rounds,
// p.round_ctas, p.rem_ctas, p.zparts and returns the grid size.
int plan_persistent(Step3dParams &p, int columns, int resident, bool in_step = false);

}  // namespace fwi
