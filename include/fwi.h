/*
 * fwi.h - C ABI of the GB300 (sm_103a) library for the hot path of acoustic
 * full-waveform inversion (FWI): forward modelling, adjoint modelling and the zero-lag
 * imaging condition that gives the gradient of the L2 misfit with respect to velocity.
 *
 * Paper: F. Huot, Y.-F. Chen, R. Clapp, C. Boneti, J. Anderson, "High-resolution
 * imaging on TPUs" (arXiv:1912.08063).  Citations below name its sections/equations:
 *   Eq. 1  phi = || d_mod - d_obs ||_2^2                          (Sec. 3)
 *   Eq. 2  P_tt = v^2 lap P + s                                   (Sec. 3)
 *   Eq. 3  P^{n+1} = -P^{n-1} + 2 P^n + v^2 dt^2 lap P^n + dt^2 s^n   (Sec. 3)
 *   Laplacian stencils of order >= 8 (8th and 16th)              (Sec. 3, Fig. 3; Sec. 4)
 *
 * Conventions for every call
 *   - Grids are C-order [nz][ny][nx] (x fastest); 2-D grids use ny = 1 and (iz, 0, ix)
 *     coordinates.  Units are SI (m, s, m/s).
 *   - Pointers marked "host or device" may point to either; the library asks the CUDA
 *     runtime which.  Host outputs make the call wait for its result; otherwise the call
 *     is asynchronous on `stream` and the caller keeps every buffer alive until the
 *     stream reaches the call.
 *   - The library owns what it allocates (velocity copy, wavefields, adjoint fields,
 *     checkpoints, traces, gradients in FP32/FP64); `fwi_destroy` frees it.  It never
 *     keeps a caller pointer past the call.
 *   - Every int-returning call returns FWI_OK (0) or a negative FWI_ERR_* code and then
 *     sets a thread-local message readable with `fwi_last_error`.  Arguments are checked
 *     on the host before any launch.  Errors detected on the device (a non-finite
 *     wavefield) are latched in the model and returned by the next call or by
 *     `fwi_sync_status`.
 *   - A model handle is not thread-safe; distinct handles are independent.
 */
#ifndef FWI_H
#define FWI_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FWI_OK            0
#define FWI_ERR_ARG      -1   /* invalid argument (shape, position, order, pointer)   */
#define FWI_ERR_CFL      -2   /* dt violates the stability limit of the scheme         */
#define FWI_ERR_OOM      -3   /* device allocation failed or budget too small          */
#define FWI_ERR_CUDA     -4   /* a CUDA runtime call or launch failed                  */
#define FWI_ERR_UNSTABLE -5   /* a wavefield became non-finite                         */
#define FWI_ERR_TIMEOUT  -6   /* a bounded device wait ran out                          */

#define FWI_SNAP_FP32 0
#define FWI_SNAP_BF16 1
#define FWI_SNAP_FP16 2

typedef struct fwi_model fwi_model;   /* opaque, library-owned */

/* Numerical options.  Zero-initialise and set what you need; zeros select defaults. */
typedef struct {
    int32_t order;              /* spatial order 2M: 8 (M = 4, default) or 16 (M = 8)  */
    int32_t nb;                 /* sponge width in cells on every face (default 20);
                                   a negative value means no sponge (closed box)        */
    int32_t snap_dtype;         /* FWI_SNAP_*: checkpoint storage type (default FP32)   */
    int32_t fold_every;         /* adjoint steps between FP32 -> FP64 gradient folds
                                   (default 256)                                        */
    int64_t snap_budget_bytes;  /* device bytes for checkpoints over all shots; 0 = a
                                   quarter of the free memory at the first gradient call;
                                   sliced as fwi_checkpoint_plan describes              */
    float   sponge_r0;          /* target reflection coefficient (default 1e-3)         */
    float   sponge_vref;        /* velocity in the sponge strength; <= 0: largest
                                   velocity of the model at creation                     */
    int32_t timing;             /* 1: bracket every time-step launch with CUDA events and
                                   accumulate kernel times (read with fwi_model_info);
                                   the call then waits for its stream at the end        */
    int32_t temporal_blocking;  /* 1: 2-D forward calls whose shots fill the GPU advance
                                   two time steps per pass (same results bit for bit;
                                   measured on GB300 within 3 % of single steps: the
                                   2-D step is latency-bound, so halving its DRAM bytes
                                   buys nothing); 2: one-shot 2-D forward calls on grids
                                   whose two states fit in the shared memory of one
                                   cluster of CTAs, with node receivers on one row,
                                   advance up to 64 steps per launch with the states on
                                   chip (same results bit for bit); other calls run
                                   single steps; default 0                              */
} fwi_opts;

/* Acquisition geometry of one call: shot s has one source and nrec receivers, each a
 * grid node (Eq. 3's point source; samples of Eq. 1's d) or, as an extension the paper
 * does not have, an off-grid position.  An off-grid point is a Kaiser-windowed sinc
 * point (Hicks 2002, Geophysics 67(1): along each axis the 8 nodes x nearest to p weigh
 * sinc(x - p) I0(6.31 sqrt(1 - ((x - p)/4)^2)) / I0(6.31), a point weighs the product
 * over axes): traces sample the weighted nodes and sources and adjoint residuals are
 * spread over the same nodes with the same weights, so injection stays the exact
 * transpose of sampling.  Its nodes must lie inside the computed grid: within the
 * physical grid, 4 cells from an edge with nb = 0, anywhere with nb >= 4.  Integer
 * positions give exactly the node results. */
typedef struct {
    int32_t nshots;
    int32_t nrec;               /* receivers per shot (>= 1)                            */
    const int32_t *src;         /* HOST [nshots][3] (iz, iy, ix) physical-grid nodes;
                                   ignored (may be NULL) when src_pos is given          */
    const int32_t *rec;         /* HOST [nshots][nrec][3]; ignored when rec_pos is given */
    const double *src_pos;      /* HOST, nullable: [nshots][3] (z, y, x) positions in
                                   physical-grid index units (fractional; y = 0 in 2-D) */
    const double *rec_pos;      /* HOST, nullable: [nshots][nrec][3]                     */
} fwi_acq;

/* Read-only facts about a model (sizes, memory and the checkpoint schedule). */
typedef struct {
    int32_t ndim, order, nb, nt;
    int64_t shape[3];           /* physical (nz, ny, nx)                                */
    int64_t computed[3];        /* with the sponge: (nz+2nb, ny+2nb or 1, nx+2nb)       */
    int64_t pitch_x;            /* floats between rows in device fields                 */
    int64_t points;             /* computed grid points per shot                        */
    int64_t device_bytes;       /* bytes the model holds on the device now              */
    int32_t snap_slots;         /* checkpoints per shot of the last gradient call       */
    int32_t shots_capacity;     /* shots the workspace is sized for                     */
    int64_t last_forward_steps; /* forward steps (incl. recomputation) of the last
                                   gradient call, per shot                              */
    int64_t last_adjoint_steps;
    int64_t last_snap_stores, last_snap_restores;
    float   sponge_eta_max[3];  /* per axis (z, y, x), 1/s                              */
    float   cfl;                /* stability number (< 1 is stable)                     */
    int64_t kernel_launches;    /* library kernel launches since creation               */
    int64_t fwd_step_launches;  /* timed forward-step launches (opts.timing), not counting
                                   those that also write a checkpoint                   */
    int64_t adj_step_launches;  /* timed reverse-step launches (opts.timing)            */
    double  fwd_step_ms;        /* their summed CUDA-event durations                    */
    double  adj_step_ms;
    int64_t store_step_launches; /* timed forward steps that also wrote a checkpoint    */
    double  store_step_ms;
    int32_t step_ctas[3];       /* 3-D models: CTAs of one persistent step launch in the
                                   forward, reverse and forward+store modes (SMs x CTAs
                                   resident per SM); 0 before the first 3-D step, and
                                   -e when the occupancy query failed with CUDA error e
                                   (the launch then uses one CTA per SM)                */
    int32_t reserved2;
} fwi_info;

/* Creates a model: the velocity grid v (physical, [nz][ny][nx] FP32, host or device,
 * copied), spacing (hz, hy, hx) in m (hy ignored in 2-D), time step dt and step count nt
 * of Eq. 3.  The computed grid adds nb sponge cells on every face of every present
 * axis, filled by edge replication of v.  Rejects with FWI_ERR_CFL when
 * v_max dt sqrt(sum_a S_M / h_a^2) / 2 >= 1, S_M being the stencil symbol at the
 * Nyquist wavenumber.  `opts` may be NULL (defaults). */
int fwi_create_model(fwi_model **out, int32_t ndim, const int64_t shape[3],
                     const float spacing[3], const float *vp, float dt, int32_t nt,
                     const fwi_opts *opts, cudaStream_t stream);

/* Replaces the velocity (same shape, host or device, copied).  The sponge strength and
 * the CFL check use the new model unless opts.sponge_vref fixed them. */
int fwi_update_velocity(fwi_model *m, const float *vp, cudaStream_t stream);

/* Forward modelling of every shot of `acq` (Eq. 2-3 with the sponge): nt steps from a
 * quiescent start, the source adds dt^2 w[n] at its node in step n, and
 *   traces[s][n][r] = u^{n+1}(rec_r)          (host or device, FP32 [nshots][nt][nrec]).
 * wavelets: FP32 [nshots][nt], host or device.  final_state (nullable, host or device)
 * receives per shot (u^nt, u^{nt-1}) on the computed grid, dense FP32
 * [nshots][2][nz_c][ny_c][nx_c]. */
int fwi_forward(fwi_model *m, const fwi_acq *acq, const float *wavelets, float *traces,
                float *final_state, cudaStream_t stream);

/* Misfit (Eq. 1, summed over shots, no 1/2) and its gradient with respect to the
 * physical velocity grid, by the exact discrete adjoint of the forward scheme and the
 * zero-lag imaging condition (gradient named in Sec. 1; the reverse recursion is the
 * transpose of the discrete forward one, so the gradient is exact for the discrete
 * misfit).  Checkpointing: binomial (revolve) schedule over nt with as many
 * checkpoints per shot as snap_budget_bytes allows (fwi_checkpoint_plan: a checkpoint is
 * u^n alone when it only ever feeds reverse steps, else the pair u^n, u^n - u^{n-1}, and
 * slots are sized by what they hold; when u^n of every step fits, nothing is
 * recomputed), stored as opts.snap_dtype with a per-checkpoint power-of-two scale;
 * forward states between checkpoints are recomputed.
 * d_obs: FP32 [nshots][nt][nrec] (host or device).  misfit: FP64 [1] (host or device,
 * nullable).  grad: FP32 physical grid (host or device, nullable).  grad64: FP64
 * physical grid (host or device, nullable).  Gradients are summed over shots. */
int fwi_adjoint_gradient(fwi_model *m, const fwi_acq *acq, const float *wavelets,
                         const float *d_obs, double *misfit, float *grad, double *grad64,
                         cudaStream_t stream);

/* Adjoint of the linear map wavelets -> traces at the model's velocity: given trace-space
 * y (FP32 [nshots][nt][nrec]) returns x (FP32 [nshots][nt]) with <F w, y> = <w, F* y>
 * up to rounding.  Host or device pointers.  Used for dot-product tests. */
int fwi_source_adjoint(fwi_model *m, const fwi_acq *acq, const float *y, float *x,
                       cudaStream_t stream);

/* phi = sum_i (d_mod[i] - d_obs[i])^2 (Eq. 1) over n FP32 samples, accumulated in FP64
 * in a fixed order (deterministic).  Device pointers; result written to misfit_dev[0].
 * Allocates its block partials with stream-ordered allocation. */
int fwi_misfit(const float *d_mod, const float *d_obs, int64_t n, double *misfit_dev,
               cudaStream_t stream);

/* The same misfit as fwi_misfit, for callers that cannot allocate device memory during
 * the call: a framework that has reserved the device's memory for its own pool, or a
 * latency-critical loop where an allocation call and its possible synchronisation are
 * not allowed.  It allocates nothing: its block partial sums live in a fixed 32 KB
 * array among the library's device globals, held by every device that loads the library
 * until the process exits.  The paper has no counterpart; this is a deployment variant.
 * Limits and rules: n <= 268435456 samples (4096 partials of 65536 samples); larger n
 * returns FWI_ERR_ARG with a message and launches nothing.  The first call on each
 * device looks up the array's device address (with that device current), so make that
 * first call before any stream capture.  All calls share the array, so calls that
 * overlap on the GPU (two streams of one device) race and must be ordered by the caller.
 * The sum is deterministic; its summation order differs from fwi_misfit's, so the two
 * agree to FP64 rounding, not bit for bit.  Device pointers; result in misfit_dev[0]. */
int fwi_misfit_noalloc(const float *d_mod, const float *d_obs, int64_t n, double *misfit_dev,
                       cudaStream_t stream);

/* Checkpoint codec (device pointers) for a state pair (a, b) = (u^n, u^{n-1}) of n FP32
 * values.  FWI_SNAP_BF16 / FWI_SNAP_FP16 store the components a and d = a - b as 16-bit
 * codes (round to nearest even), each after scaling by its own
 * s = 2^floor(log2(T / max|component|)), T = 2^14 for FP16 and 1 for BF16 (s = 1 for an
 * all-zero component): code holds [2][n] 16-bit values, scale[0..1] receive (s_a, s_d).
 * FWI_SNAP_FP32 copies a and b ([2][n] FP32, scales 1).  Non-finite input sets the
 * scales to NaN and returns FWI_OK (the codes are then unspecified).  Allocates two
 * words of stream-ordered scratch. */
int fwi_snapshot_encode(const float *a, const float *b, int64_t n, int32_t dtype,
                        void *code, float *scale, cudaStream_t stream);
/* Inverse of fwi_snapshot_encode: a = code[0] / s_a, b = a - code[1] / s_d. */
int fwi_snapshot_decode(const void *code, const float *scale, int64_t n, int32_t dtype,
                        float *a, float *b, cudaStream_t stream);

/* Host only.  Binomial checkpointing schedule (Griewank-Walther revolve) for the reverse
 * sweep of nsteps forward steps with nslots checkpoints besides the zero initial state.
 * Writes up to max_actions actions as int32 pairs (kind, arg):
 *   kind 1 ADVANCE  arg = number of forward steps from the current state
 *   kind 2 STORE    arg = slot (0..nslots-1) receiving the current state
 *   kind 3 RESTORE  arg = slot, or -1 for the zero initial state
 *   kind 4 ADJOINT  arg = m: one reverse step that needs the state after m steps
 * Adjoint steps run for m = nsteps down to 1.  *n_actions and *n_forward receive the
 * action count and the number of forward steps (the minimum for nslots).  Returns
 * FWI_ERR_ARG when max_actions is too small (n_actions still receives the need). */
int fwi_revolve_schedule(int32_t nsteps, int32_t nslots, int32_t *actions,
                         int64_t max_actions, int64_t *n_actions, int64_t *n_forward);

/* Host only.  The checkpoint plan a gradient call makes for nsteps steps from a budget
 * of half_slots units, one unit being the codes of one field (all shots): a checkpoint
 * restored only for its reverse step is u^n alone (one unit), any other the pair
 * u^n, u^n - u^{n-1} (two units), and a slot takes two units if the revolve schedule
 * ever stores a pair in it.  The plan is the largest slot count whose layout fits:
 * *slots, *pair_slots (slots of two units) and *n_forward (forward steps of the
 * schedule; nsteps when u^n of every step fits, i.e. no recomputation).  FWI_ERR_ARG
 * for nsteps < 1 or half_slots < 0. */
int fwi_checkpoint_plan(int32_t nsteps, int64_t half_slots, int32_t *slots,
                        int32_t *pair_slots, int64_t *n_forward);

/* Host only.  Central second-derivative weights c_0..c_M of order 2M (M = order/2) as
 * FP64 (the stencil of Eq. 2-3's Laplacian). */
int fwi_fd_coeffs(int32_t order, double *c);

/* Host only.  Stability number v_max dt sqrt(sum_a S_M/h_a^2)/2 of the leapfrog. */
double fwi_cfl_number(int32_t ndim, int32_t order, const float spacing[3], float vmax,
                      float dt);

int fwi_model_info(const fwi_model *m, fwi_info *out);

/* ------------------------------------------------------------------ serving loop
 * Continuous batching of independent forward and gradient requests on one GPU (a
 * systems pattern around the paper's method: each request is one shot of Eq. 2-3 or
 * one misfit gradient on its own grid).  Requests are admitted in arrival order as soon
 * as they have arrived, a slot is free and their device-memory estimate fits in the
 * budget's remainder; an admitted request owns a model (wavefields and checkpoints stay
 * on the device) and a stream, and one host thread issues the admitted requests' time
 * steps round-robin (steps_per_turn at a time, at most two turns in flight per request),
 * so their work overlaps on the device.  2-D forward requests with node source and
 * receivers share one launch instead: each tick, one captured graph of persistent
 * multi-request step and sampling kernels advances all of them by steps_per_turn
 * (rounded up to even) steps from a device table of request descriptors updated in
 * place; requests small enough to keep both states in the shared memory of one cluster
 * of CTAs are advanced by a single launch per tick that runs all those steps on chip.
 * Finished requests are retired and release their memory.  max_active = 1
 * serves one request at a time on the same kernels. */
#define FWI_REQ_FORWARD  0
#define FWI_REQ_GRADIENT 1

typedef struct {
    int32_t kind;               /* FWI_REQ_FORWARD or FWI_REQ_GRADIENT                  */
    int32_t ndim;
    int64_t shape[3];           /* physical (nz, ny, nx), ny = 1 in 2-D                 */
    float   spacing[3];
    float   dt;
    int32_t nt;
    int32_t order;              /* 8 or 16                                              */
    int32_t snap_dtype;         /* checkpoint storage of gradient requests (FWI_SNAP_*) */
    int32_t nrec;
    int32_t src[3];             /* (iz, iy, ix)                                         */
    int32_t reserved;
    const float   *vp;          /* HOST physical velocity                               */
    const float   *wavelet;     /* HOST [nt]                                            */
    const int32_t *rec;         /* HOST [nrec][3]                                       */
    const float   *d_obs;       /* HOST [nt][nrec] (gradient requests)                  */
    float         *traces_out;  /* HOST [nt][nrec] (forward requests), nullable         */
    float         *grad_out;    /* HOST physical grid (gradient requests), nullable     */
    double  arrival;            /* seconds after the start of fwi_serve                 */
} fwi_request;

typedef struct {
    int32_t status;             /* FWI_OK or the request's error code                   */
    int32_t shared_launch;      /* 0: own stream; 1: shared launch of multi-request
                                   step kernels; 2: shared cluster launch, k steps per
                                   launch with the states in shared memory            */
    double  misfit;             /* gradient requests (Eq. 1)                            */
    double  t_admit, t_start, t_done;   /* seconds after the start of fwi_serve         */
    int64_t device_bytes;       /* device memory the request's model held at admission  */
    int64_t reserved_bytes;     /* what admission reserved for it from the budget       */
} fwi_result;

typedef struct {
    int64_t hbm_budget_bytes;   /* device memory for admitted requests (0: 80 % free)   */
    int32_t max_active;         /* admitted requests at once (default 16)               */
    int32_t steps_per_turn;     /* time steps issued per request per turn (default 8)   */
    int32_t snap_slots;         /* checkpoint budget per gradient request, in pairs
                                   (default 64; slots holding u^n alone take half)      */
    int32_t nb;                 /* sponge width (default 20)                            */
    int32_t no_shared_launch;   /* 1: every request issues its own steps on its own
                                   stream; 0 (default): 2-D forward requests with node
                                   source and receivers are advanced together by the
                                   shared launch (one graph of multi-request step and
                                   sampling kernels per tick over a device table of
                                   request descriptors)                                */
} fwi_serve_opts;

/* Runs the request stream to completion: waits for each arrival time, admits, steps and
 * retires requests; results[i] belongs to reqs[i].  The host buffers of every request
 * must stay valid for the whole call.  Returns FWI_OK once every request has a status
 * (per-request failures are reported in results[i].status). */
int fwi_serve(const fwi_request *reqs, int32_t n, const fwi_serve_opts *opts,
              fwi_result *results);

/* Failure-path self-test of the bounded device waits (no counterpart in the paper; the
 * waits guard the TMA-staged 3-D step kernels).  Launches, on `stream`, one CTA that arms
 * an mbarrier the way the step kernels' producer does (an arrival with an expected
 * transaction count), issues no copy, and waits with the step kernels' bounded wait
 * limited to `polls` polls (1 <= polls <= 2^22).  The wait runs out and raises the model's
 * latched timeout status exactly as a step kernel whose data never arrived would: the
 * next fwi_sync_status returns FWI_ERR_TIMEOUT, and every later call on this model
 * returns it too (the status stays latched; create a new model to continue).  No copy is
 * in flight, so nothing faults and nothing waits without bound.  Returns FWI_ERR_ARG for
 * polls out of range, FWI_ERR_CUDA if the launch fails. */
int fwi_selftest_wait(fwi_model *m, int32_t polls, cudaStream_t stream);

/* Waits for the model's last stream and returns its latched device status. */
int fwi_sync_status(fwi_model *m);

void fwi_destroy(fwi_model *m);

/* Message of the last error on this thread ("" if none). */
const char *fwi_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FWI_H */
