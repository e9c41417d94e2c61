// Internal types shared by the CUDA kernels and the host executor of libfwi.
// Nothing here is part of the C ABI (include/fwi.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace fwi {

constexpr int kMaxM = 8;   // stencil radius of the 16th-order Laplacian

// Device layout of one shot's field on the computed grid (sponge included):
// C-order [nz][ny][px] FP32, rows padded to px floats (a multiple of 8, so every row
// starts on a 16-byte boundary in FP32 and in the 16-bit checkpoint codes), shots
// `field` floats apart (a multiple of 64).
// Columns nx..px-1 are zero and never written.
struct Geom {
    int ndim;       // 2 or 3
    int M;          // stencil radius
    int nz, ny, nx; // computed extents (ny = 1 in 2-D)
    int px;         // row pitch in floats
    int64_t plane;  // ny * px
    int64_t field;  // floats per shot
};

// Second-derivative weights c_k / h_a^2 per axis, k = 0..M, and the combined centre
// weight c_0 * sum_a 1/h_a^2.
struct Coefs {
    float cz[kMaxM + 1];
    float cy[kMaxM + 1];
    float cx[kMaxM + 1];
    float c0;
};

// One time step of the damped leapfrog on every shot of a batch:
//   out = (2 cur + W (L cur) - (1 - s) prev + [dt^2 w[n] at the source]) / (1 + s),
//   s = sig_z[z] + sig_y[y] + sig_x[x]  (= eta dt / 2),
// written over `prev`.  The reverse step with imaging (cur = mu^{m+1}, aux = u^m) adds
// no source to `out` and accumulates the transposed zero-lag imaging term
//   gacc += aux * (L cur),   at the source point  gacc -= dt^2 w[n] cur / W
// (the receiver term of the same sum is added once from the traces: launch_rec_image).
struct StepParams {
    Geom g;
    Coefs c;
    const float *cur;
    float *prev;
    const float *W;
    const float *sig_z, *sig_y, *sig_x;
    const int64_t *src_off;   // [nshots] offsets within a shot's field, or nullptr
    const float *wavelet;     // [nshots][nt]
    int nt, n;
    const int *n_dev;         // nullable: the step index is *n_dev + n (a captured CUDA graph
                              // replays its steps with a device-side step counter)
    float dt2;
    // imaging only: u^m, an FP32 field (aux_fmt 0, aux_scale null) or the first component
    // of a checkpoint slot read in place (aux_fmt = its FWI_SNAP_* type, u^m = code /
    // scale, bit for bit what the decode kernel would write)
    const void *aux;
    int aux_fmt;              // 0 FP32, 1 BF16, 2 FP16
    int64_t aux_stride;       // elements per shot
    const float *aux_scale;   // per shot at [2 s], or nullptr (scale 1)
    float *gacc;              // imaging only: gradient accumulator
    int zchunk;               // planes per CTA along z
    int nzchunks;
    // nullable, 3-D forward step only: a checkpoint store of this step's input pair
    // (cur = u^n, prev = u^{n-1}) written from the epilogue before prev is overwritten, in
    // the encode kernel's format (component a = u^n, d = u^n - u^{n-1}, or the FP32 pair)
    void *st_code;
    const float *st_scale;    // per shot at [2s] (a) and [2s+1] (d), set by launch_snap_scales
    int st_dtype, st_comps;
    int64_t st_cstride;       // code elements per shot (both components)
    unsigned *maxbits;        // nullable, forward step only: per shot, raise [2s] / [2s+1]
                              // to the bits of max|out| / max|out - cur| (the checkpoint
                              // codec's scales of the new state pair)
    unsigned *err;            // TMA-staged kernels: status word, bit 1 (value 2) = a
                              // bounded wait gave up
    // 3-D receivers sampled / residuals injected in the step's epilogue (set by the
    // library when every receiver is a node of one plane): forward steps write
    // rec_tr[s][n][r] = u^{n+1}(rec_r); reverse steps add inj_scale[s][r] inj_q[s][inj_n][r]
    // to mu^m at the receivers (nullptr: the separate kernels do it)
    float *rec_tr;
    const float *inj_q, *inj_scale;
    int inj_n;
};

// An off-grid source or receiver (Kaiser-windowed sinc point): taps at the computed-grid
// nodes (z0 + a, y0 + b, x0 + c), a, c < kTaps, b < kTaps in 3-D (b = 0 in 2-D), with
// weight w[a] * w[kTaps + b] * w[2 kTaps + c].
constexpr int kTaps = 8;
struct PointTaps {
    int32_t z0, y0, x0, pad;
    float w[3 * kTaps];
};

// ---- off-grid points (k_points.cu) ----
cudaError_t launch_sample_pts(const Geom &g, const float *f, const PointTaps *pts, int nshots,
                              int nrec, int nt, int n, float *traces, cudaStream_t s,
                              const int *n_dev = nullptr);
// kind 0: f += dt^2 q[s][n] wt / a+ (source; q = wavelets, per_shot = 1);
// kind 1: f += factor (W / a+) wt q[s][n][r] (adjoint injection; per_shot = nrec)
cudaError_t launch_inject_pts(const Geom &g, float *f, const PointTaps *pts, int npts,
                              int per_shot, const float *W, const float *sig_z,
                              const float *sig_y, const float *sig_x, const float *q, int nt,
                              int n, float dt2, float factor, int kind, cudaStream_t s,
                              const int *n_dev = nullptr);
// transposed-imaging point terms: kind 0 g -= dt^2 q[s][n] wt x / W (x = mu^{m+1});
// kind 1 g += 2 wt x q[s][n][r] (x = u^m as FP32 or a 16-bit code, see StepParams::aux)
cudaError_t launch_image_pts(const Geom &g, float *gacc, const void *x, int xfmt,
                             int64_t xstride, const float *xscale, const PointTaps *pts,
                             int npts, int per_shot, const float *W, const float *q, int nt,
                             int n, float dt2, int kind, cudaStream_t s);
// x[s][n] = dt^2 sum_t wt f[t] / W[t]
cudaError_t launch_gather_src_pts(const Geom &g, const float *f, const PointTaps *pts,
                                  int nshots, const float *W, float dt2, int nt, int n,
                                  float *x, cudaStream_t s);

// 2-D step (k_step2d.cu); the 3-D step has its own launcher (step3d.h)
cudaError_t launch_step2d(const StepParams &p, int nshots, bool imaging, cudaStream_t s);

// The serving loop's shared 2-D forward launch: a device table of requests, each a
// one-shot 2-D forward run with a node source and node receivers.  A tick of k steps is
// k launches of each kernel (step t = 0 .. k - 1).
struct Batch2dEntry {
    StepParams p;             // the request's step parameters (g, c, W, sig, src_off,
                              // wavelet, nt, dt2, zchunk, nzchunks; cur/prev/n unused)
    float *u0, *u1;           // u^{n0} and u^{n0 - 1} at the tick's start
    int n0;                   // step index at the tick's start
    int xtiles;               // work items: xtiles x p.nzchunks
    int work0, rec0;          // first work item and first receiver of the entry
    const int64_t *rec_off;   // [nrec] receiver offsets in the field
    float *traces;            // [nt][nrec]
    int nrec;
    int nsamp;                // receivers the sampling kernel reads: nrec, or 0 when the
                              // step samples them (rec_z >= 0)
    int rec_z, rec_x0;        // receivers on row rec_z, columns rec_x0 .. rec_x0 + nrec - 1
                              // (rec_z = -1: any other layout)
    int pad[2];
};
constexpr int kBatch2dMax = 64;
struct Batch2d {
    int count, total_work, total_rec, pad;   // total_rec: receivers of the sampling kernel
    Batch2dEntry e[kBatch2dMax];
};
// Persistent grid of k_step2d_multi for radius M (resident CTAs on the current device).
int multi2d_grid(int M);
cudaError_t launch_step2d_multi(const Batch2d *tab, int M, int t, int grid, cudaStream_t s);
cudaError_t launch_sample_multi(const Batch2d *tab, int t, int grid, cudaStream_t s);
// Temporal blocking on chip: k steps of every request of the table in one launch, one
// cluster of C CTAs per request, each CTA holding a band of rows of both states in shared
// memory (smem bytes per CTA: 2 ceil(nz / C) px floats of the largest request).  For
// requests with receivers on one row (rec_z >= 0) and nz / C > M.
// cluster2d_size: the cluster size to use (16, else 8; 0 if clusters cannot be launched).
int cluster2d_size(int M);
int cluster2d_max_smem();
cudaError_t launch_step2d_cluster(const Batch2d *tab, int M, int k, int C, int nreq, int smem,
                                  cudaStream_t s);
// Two forward steps in one pass (2-D): from (p.cur = u^n, p.prev = u^{n-1}) write u^{n+1}
// to out1 and u^{n+2} to out2 (neither may alias cur or prev); sources at steps n and
// n + 1.  step2d_tb2_chunks is 0 when the batch is too small to fill the GPU (then use
// single steps); the launcher picks its own strips and z-chunks.
int step2d_tb2_chunks(const Geom &g, int nshots);
cudaError_t launch_step2d_tb2(const StepParams &p, int nshots, float *out1, float *out2,
                              int nchunks, cudaStream_t s);

// ---- auxiliary kernels (k_aux.cu) ----
cudaError_t launch_build_W(const Geom &g, int nb, const int64_t np[3], const float *v,
                           float dt, float *W, cudaStream_t s);
// gacc64[rec] += 2 sum_k d[k] (d[k] - dobs[k]) per receiver: the receiver term of the
// transposed imaging sum (traces d[shot][k][rec] hold u^{k+1} at the receivers)
cudaError_t launch_rec_image(const Geom &g, const float *d, const float *dobs,
                             const int64_t *rec_off, int nshots, int nrec, int nt,
                             double *gacc64, cudaStream_t s);
// gacc64[src] -= dt^2 w[0] mu1[src] / W[src] per shot: the m = 0 source term of the same
// sum (no reverse step runs at m = 0)
cudaError_t launch_src_image(const Geom &g, const float *mu1, const int64_t *src_off,
                             const float *W, const float *wavelet, float dt2, int nshots,
                             int nt, double *gacc64, cudaStream_t s);
// n_dev (nullable): the trace row is *n_dev + n
cudaError_t launch_sample(const Geom &g, const float *field, const int64_t *rec_off,
                          int nshots, int nrec, int nt, int n, float *traces,
                          cudaStream_t s, const int *n_dev = nullptr);
// *counter += add (one thread; the step counter of a captured graph)
cudaError_t launch_tick(int *counter, int add, cudaStream_t s);
// *counter = value
cudaError_t launch_set_counter(int *counter, int value, cudaStream_t s);
cudaError_t launch_inject(const Geom &g, float *field, const int64_t *rec_off,
                          const float *scale, const float *q, int nshots, int nrec, int nt,
                          int sample, cudaStream_t s);
cudaError_t launch_gather_src(const Geom &g, const float *field, const int64_t *src_off,
                              const float *src_scale, int nshots, int nt, int sample,
                              float *x, cudaStream_t s);
cudaError_t launch_rec_scale(const Geom &g, const float *W, const float *sig_z,
                             const float *sig_y, const float *sig_x, const int64_t *off,
                             int count, float factor, int mode, float *out, cudaStream_t s);
// residual r = d - d_obs in place of d (when store_r) and block partials of sum r^2
// (flag, when given, is raised if the sum is not finite)
cudaError_t launch_misfit(const float *d, const float *dobs, float *r_out, int64_t n,
                          double *partials, int nblocks, double *result, unsigned *flag,
                          cudaStream_t s);
int misfit_blocks(int64_t n);
// per shot: scale[2s], scale[2s+1] from maxbits as the encode kernel derives them (flag
// raised for a non-finite maximum)
cudaError_t launch_snap_scales(const unsigned *maxbits, int nshots, int dtype, float *scale,
                               unsigned *flag, cudaStream_t s);
cudaError_t launch_maxabs(const float *a, const float *b, int64_t n, int64_t stride,
                          int nshots, unsigned *maxbits, cudaStream_t s);
// comps = 2: the pair (a, b); comps = 1: a only (a checkpoint restored only for imaging)
cudaError_t launch_encode(const float *a, const float *b, int64_t n, int64_t stride,
                          int nshots, int dtype, const unsigned *maxbits, void *code,
                          int64_t code_stride, float *scale, unsigned *flag, int comps,
                          cudaStream_t s);
cudaError_t launch_decode(const void *code, int64_t code_stride, const float *scale,
                          int64_t n, int64_t stride, int nshots, int dtype, float *a, float *b,
                          int comps, cudaStream_t s);
cudaError_t launch_fold(float *g32, double *g64, int64_t n, cudaStream_t s);
cudaError_t launch_finish(const Geom &g, int nb, const int64_t np[3], int nshots,
                          const double *g64, const float *v, float *grad32, double *grad64,
                          cudaStream_t s);
// One CTA that arms an mbarrier with an expected byte count, issues no copy and waits with
// the step kernels' bounded wait limited to `polls`; raises bit 1 of *err when it runs
// out (k_selftest.cu)
cudaError_t launch_wait_selftest(unsigned *err, int polls, cudaStream_t s);
cudaError_t launch_nonfinite_check(const float *a, int64_t n, unsigned *flag,
                                   cudaStream_t s);

}  // namespace fwi
