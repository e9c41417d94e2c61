// Serving loop: continuous batching of forward and gradient requests on one GPU.
//
// Requests arrive over time (each carries its own grid, velocity, acquisition and, for a
// gradient, observed traces).  A request is admitted, in arrival order, as soon as it
// has arrived, a slot is free and its device-memory estimate fits in what the budget has
// left; it then owns a model (wavefields and checkpoints stay on the device) and a CUDA
// stream of its own.  One host thread issues the admitted requests' work round-robin, a
// few time steps per turn and at most two turns in flight per request, so requests of
// different sizes and phases (forward sweep, recomputation, reverse sweep) overlap on
// the device.  A request that has issued its last step gets its result copies queued;
// when they land it is retired, its memory returns to the budget and the next waiting
// request can be admitted.  max_active = 1 gives the one-request-at-a-time baseline on
// the same kernels.
//
// Shared launch: 2-D forward requests (one shot, node source and receivers) of the same
// stencil radius do not issue their own steps.  They join a pool whose device table holds
// one descriptor per request (its step parameters, state buffers, step index, receivers
// and traces); each tick, the loop refreshes the table in place (one upload from pinned
// memory on the pool's stream) and replays one captured graph of k persistent launches
// of the multi-request step kernel and k of the multi-request sampling kernel, which
// advance every pooled request by k steps.  The graph reads the table at run time, so
// admissions and retirements change only the table, never the graph.  A request that
// reaches its last step leaves the pool: its own stream waits for that tick before the
// result copies.  Small requests (both states fit in the shared memory of one cluster
// of CTAs) go to cluster pools instead, whose tick is a single launch that advances each
// request by k steps with its states on chip (temporal blocking, k_step2d_cluster).
#include <algorithm>
#include <chrono>
#include <cstddef>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "fwi.h"

#include "fwi_internal.h"

namespace fwi {
struct Job;
bool job_batchable(const Job *j);
int job_batch_entry(Job *j, Batch2dEntry *e, int zchunk);
int job_batch_moved(Job *j, int steps, bool *done);
Job *job_forward(fwi_model *m, const fwi_acq *acq, const float *wavelets, cudaStream_t s, int *rc);
Job *job_gradient(fwi_model *m, const fwi_acq *acq, const float *wavelets, const float *d_obs,
                  cudaStream_t s, int *rc);
int job_advance(Job *j, int64_t units, bool *done);
int job_finish(Job *j, double *misfit_host, float *out_host);
void job_free(Job *j);
int report_error(int code, const std::string &msg);
}  // namespace fwi

namespace {

using clk = std::chrono::steady_clock;

struct Slot {
    int req = -1;
    fwi_model *model = nullptr;
    cudaStream_t stream = nullptr;
    fwi::Job *job = nullptr;
    cudaEvent_t turn = nullptr;   // recorded after each turn's launches
    cudaEvent_t done = nullptr;   // recorded after the result copies
    bool issued_all = false, finishing = false;
    int64_t bytes = 0;
    fwi_acq acq{};
    float *out_pinned = nullptr;  // traces or gradient
    double *misfit_pinned = nullptr;
    size_t out_bytes = 0;
    int pool = -1;                // index of the shared-launch pool it is in, or -1
    bool pool_synced = false;     // the pool's stream has waited for its set-up
};

// A pool of requests advanced together by the shared launch.  kind 0: per tick, k
// launches of the multi-request step kernel (and of the sampling kernel); kind 1: per
// tick, one launch of the cluster kernel, which advances each request by k steps with
// its states held in the shared memory of one cluster of C CTAs (small grids only).
struct Pool {
    int kind = 0, C = 0;
    int M = 0;
    fwi::Batch2d *dev = nullptr;       // device table
    fwi::Batch2d *host[2] = {};        // pinned staging, used alternately
    cudaEvent_t uploaded[2] = {};      // the upload from host[i] has finished
    bool pending[2] = {false, false};
    int buf = 0;
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr;       // one tick: k x (multi step, multi sample)
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaGraphNode_t> nodes;   // its kernel nodes in launch order
    std::vector<cudaKernelNodeParams> params;
    int grid_step = 0, grid_sample = 0;   // persistent grids (resident CTAs)
    bool sampling = true;                 // the sampling nodes are enabled
    int k = 0;
    cudaEvent_t tick = nullptr;        // recorded after a tick that finished a request
    std::vector<int> members;          // slot indices
    bool failed = false;               // set-up failed: requests run on their own streams
};

constexpr int kPoolZChunk = 128;   // most rows per work item of the multi-request step
constexpr int kPools = 4;          // shared-launch pools per stencil radius
// Cluster pools take grids of at most this many computed points (measured on GB300: one
// request alone runs 4.3x / 2.3x / 1.3x faster on chip than in single steps at 128^2 /
// 256^2 / 384^2, and no faster from about 512^2 on) and advance them by at least
// kClusterTick steps per tick (the states stay on chip for the whole launch).
constexpr int64_t kClusterMaxPoints = 200000;
constexpr int kClusterTick = 64;

void pool_release(Pool &p)
{
    if (p.stream) cudaStreamSynchronize(p.stream);
    if (p.exec) cudaGraphExecDestroy(p.exec);
    if (p.graph) cudaGraphDestroy(p.graph);
    for (int i = 0; i < 2; ++i) {
        if (p.host[i]) cudaFreeHost(p.host[i]);
        if (p.uploaded[i]) cudaEventDestroy(p.uploaded[i]);
    }
    if (p.tick) cudaEventDestroy(p.tick);
    if (p.dev) cudaFree(p.dev);
    if (p.stream) cudaStreamDestroy(p.stream);
    p = Pool();
}

// Allocates the pool's table and stream and captures its tick graph (k steps).
int pool_setup(Pool &p, int kind, int M, int k, int C)
{
    p.kind = kind;
    p.C = C;
    p.M = M;
    p.k = k;
    cudaError_t e = cudaStreamCreateWithFlags(&p.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc((void **)&p.dev, sizeof(fwi::Batch2d));
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        e = cudaMallocHost((void **)&p.host[i], sizeof(fwi::Batch2d));
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p.uploaded[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p.tick, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemsetAsync(p.dev, 0, sizeof(fwi::Batch2d), p.stream);
    if (e != cudaSuccess) return fwi::report_error(FWI_ERR_CUDA, std::string("serve pool: ") + cudaGetErrorString(e));
    p.grid_step = kind == 0 ? fwi::multi2d_grid(M) : 0;
    p.grid_sample = 152 * 4;
    const size_t want = kind == 0 ? (size_t)(2 * k) : 1;
    e = cudaStreamBeginCapture(p.stream, cudaStreamCaptureModeThreadLocal);
    if (kind == 0) {
        for (int t = 0; t < k && e == cudaSuccess; ++t) {
            e = fwi::launch_step2d_multi(p.dev, M, t, p.grid_step, p.stream);
            if (e == cudaSuccess) e = fwi::launch_sample_multi(p.dev, t, p.grid_sample, p.stream);
        }
    } else {
        e = fwi::launch_step2d_cluster(p.dev, M, k, C, 1, fwi::cluster2d_max_smem(), p.stream);
    }
    const cudaError_t ec = cudaStreamEndCapture(p.stream, &p.graph);
    if (e == cudaSuccess) e = ec;
    // the kernel nodes, in launch order (a chain), so each tick can size their grids
    size_t nn = 0;
    if (e == cudaSuccess) e = cudaGraphGetNodes(p.graph, nullptr, &nn);
    if (e == cudaSuccess && nn != want) e = cudaErrorInvalidValue;
    if (e == cudaSuccess) {
        std::vector<cudaGraphNode_t> all(nn);
        e = cudaGraphGetRootNodes(p.graph, all.data(), &nn);
        cudaGraphNode_t cur = nn == 1 ? all[0] : nullptr;
        while (e == cudaSuccess && cur) {
            p.nodes.push_back(cur);
            cudaKernelNodeParams kp{};
            e = cudaGraphKernelNodeGetParams(cur, &kp);
            p.params.push_back(kp);
            size_t ne = 0;
            if (e == cudaSuccess) e = cudaGraphNodeGetDependentNodes(cur, nullptr, nullptr, &ne);
            cudaGraphNode_t nx = nullptr;
            if (e == cudaSuccess && ne == 1) e = cudaGraphNodeGetDependentNodes(cur, &nx, nullptr, &ne);
            cur = ne == 1 ? nx : nullptr;
        }
        if (e == cudaSuccess && p.nodes.size() != want) e = cudaErrorInvalidValue;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p.exec, p.graph, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fwi::report_error(FWI_ERR_CUDA, std::string("serve pool graph: ") + cudaGetErrorString(e));
    }
    return FWI_OK;
}

int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// Device bytes a request will hold: the model's fields, traces, staging and checkpoints.
int64_t estimate_bytes(const fwi_request &r, int nb, int snap_slots)
{
    const int64_t nz = r.shape[0] + 2 * nb, ny = r.ndim == 3 ? r.shape[1] + 2 * nb : 1,
                  nx = r.shape[2] + 2 * nb;
    const int64_t field = round_up(nz * ny * round_up(nx, 8), 64) * 4;
    const int64_t phys = r.shape[0] * r.shape[1] * r.shape[2] * 4;
    const int64_t traces = (int64_t)r.nt * r.nrec * 4;
    int64_t b = field + 2 * phys + 2 * traces + (int64_t)r.nt * 4 + (8 << 20);
    if (r.kind == FWI_REQ_FORWARD) return b + 2 * field;
    const int esz = r.snap_dtype == FWI_SNAP_FP32 ? 4 : 2;
    // u pair, mu pair, FP32 and FP64 gradients, observed traces, checkpoints
    return b + 7 * field + traces + (int64_t)snap_slots * 2 * (field / 4) * esz;
}

int release(Slot &s)
{
    if (s.job) fwi::job_free(s.job);
    if (s.model) fwi_destroy(s.model);
    if (s.turn) cudaEventDestroy(s.turn);
    if (s.done) cudaEventDestroy(s.done);
    if (s.stream) cudaStreamDestroy(s.stream);
    if (s.out_pinned) cudaFreeHost(s.out_pinned);
    if (s.misfit_pinned) cudaFreeHost(s.misfit_pinned);
    s = Slot();
    return FWI_OK;
}

// Creates the request's model, stream and job.
int admit(Slot &s, int idx, const fwi_request &r, const fwi_serve_opts &o)
{
    s.req = idx;
    cudaError_t e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.turn, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
    if (e != cudaSuccess)
        return fwi::report_error(FWI_ERR_CUDA, std::string("serve: ") + cudaGetErrorString(e));
    fwi_opts mo{};
    mo.order = r.order;
    mo.nb = o.nb;
    mo.snap_dtype = r.snap_dtype;
    const int esz = r.snap_dtype == FWI_SNAP_FP32 ? 4 : 2;
    const int64_t nz = r.shape[0] + 2 * o.nb, ny = r.ndim == 3 ? r.shape[1] + 2 * o.nb : 1,
                  nx = r.shape[2] + 2 * o.nb;
    mo.snap_budget_bytes = (int64_t)o.snap_slots * 2 * round_up(nz * ny * round_up(nx, 8), 64) * esz;
    if (mo.snap_budget_bytes <= 0) mo.snap_budget_bytes = 1;
    int rc = fwi_create_model(&s.model, r.ndim, r.shape, r.spacing, r.vp, r.dt, r.nt, &mo,
                              s.stream);
    if (rc != FWI_OK) return rc;
    s.acq.nshots = 1;
    s.acq.nrec = r.nrec;
    s.acq.src = r.src;
    s.acq.rec = r.rec;
    if (r.kind == FWI_REQ_FORWARD) {
        s.out_bytes = (size_t)r.nt * r.nrec * sizeof(float);
        s.job = fwi::job_forward(s.model, &s.acq, r.wavelet, s.stream, &rc);
    } else {
        s.out_bytes = (size_t)r.shape[0] * r.shape[1] * r.shape[2] * sizeof(float);
        s.job = fwi::job_gradient(s.model, &s.acq, r.wavelet, r.d_obs, s.stream, &rc);
    }
    if (rc != FWI_OK) return rc;
    e = cudaMallocHost((void **)&s.out_pinned, s.out_bytes);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&s.misfit_pinned, sizeof(double));
    if (e != cudaSuccess)
        return fwi::report_error(FWI_ERR_OOM, std::string("serve: pinned buffer: ") +
                                                  cudaGetErrorString(e));
    return FWI_OK;
}

}  // namespace

extern "C" int fwi_serve(const fwi_request *reqs, int32_t n, const fwi_serve_opts *opts,
                         fwi_result *results)
{
    if (!reqs || !results || n < 0) return fwi::report_error(FWI_ERR_ARG, "serve: bad arguments");
    fwi_serve_opts o{};
    if (opts) o = *opts;
    if (o.max_active <= 0) o.max_active = 16;
    if (o.steps_per_turn <= 0) o.steps_per_turn = 8;
    if (o.snap_slots <= 0) o.snap_slots = 64;
    if (o.nb == 0) o.nb = 20;
    if (o.hbm_budget_bytes <= 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        o.hbm_budget_bytes = (int64_t)(fr * 0.8);
    }
    for (int i = 0; i < n; ++i) {
        std::memset(&results[i], 0, sizeof(fwi_result));
        results[i].status = 1;   // pending
    }
    // arrival order
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return reqs[a].arrival < reqs[b].arrival; });

    std::vector<Slot> slots(o.max_active);
    // shared-launch pools, radius 4 and radius 8, set up on first use; a tick is an even
    // number of steps (steps_per_turn rounded up)
    // kPools pools per radius, filled round-robin: their ticks overlap on the device
    // (measured on GB300: one pool serialises its requests' steps behind one another,
    // four match the throughput of one stream per request)
    // pools: [kind][radius 4, 8][kPools]
    std::vector<Pool> pools(2 * 2 * kPools);
    int rr = 0;
    int cl_size[2] = {-1, -1};   // cluster size per radius (0: no cluster pools)
    const int tick_k = (o.steps_per_turn + 1) / 2 * 2;
    const bool share = o.no_shared_launch == 0;
    int64_t used = 0;
    size_t next = 0;
    int finished = 0;
    const auto t0 = clk::now();
    auto now = [&]() { return std::chrono::duration<double>(clk::now() - t0).count(); };

    while (finished < n) {
        // admission, in arrival order
        while (next < order.size()) {
            const int idx = order[next];
            const fwi_request &r = reqs[idx];
            if (r.arrival > now()) break;
            const int64_t est = estimate_bytes(r, o.nb, o.snap_slots);
            if (est > o.hbm_budget_bytes) {   // can never fit
                results[idx].status = FWI_ERR_OOM;
                results[idx].t_done = now();
                ++next;
                ++finished;
                continue;
            }
            Slot *free_slot = nullptr;
            for (auto &s : slots)
                if (s.req < 0) {
                    free_slot = &s;
                    break;
                }
            if (!free_slot || used + est > o.hbm_budget_bytes) break;
            results[idx].t_admit = now();
            const int rc = admit(*free_slot, idx, r, o);
            if (rc != FWI_OK) {
                results[idx].status = rc;
                results[idx].t_done = now();
                release(*free_slot);
                ++next;
                ++finished;
                continue;
            }
            if (share && fwi::job_batchable(free_slot->job)) {
                const int M = r.order / 2, ri = r.order == 16 ? 1 : 0;
                if (cl_size[ri] < 0) cl_size[ri] = fwi::cluster2d_size(M);
                // small grids whose receivers form one row go to the cluster pools
                fwi::Batch2dEntry probe;
                int kind = 0;
                const int C = cl_size[ri];
                if (C > 0 && fwi::job_batch_entry(free_slot->job, &probe, 64) == FWI_OK &&
                    probe.rec_z >= 0 && probe.p.g.nz / C > M &&
                    (int64_t)probe.p.g.nz * probe.p.g.px <= kClusterMaxPoints &&
                    2LL * ((probe.p.g.nz + C - 1) / C) * probe.p.g.px * 4 <= fwi::cluster2d_max_smem())
                    kind = 1;
                const int pi = (kind * 2 + ri) * kPools + (rr++ % kPools);
                Pool &pl = pools[pi];
                if (!pl.stream && !pl.failed &&
                    pool_setup(pl, kind, M, kind ? std::max(tick_k, kClusterTick) : tick_k, C) != FWI_OK) {
                    pool_release(pl);
                    pl.failed = true;
                }
                if (!pl.failed && (int)pl.members.size() < fwi::kBatch2dMax &&
                    cudaEventRecord(free_slot->turn, free_slot->stream) == cudaSuccess) {
                    free_slot->pool = pi;   // its set-up is ordered before the pool's next tick
                    results[idx].shared_launch = 1 + kind;
                    pl.members.push_back((int)(free_slot - slots.data()));
                } else {
                    cudaGetLastError();
                }
            }
            free_slot->bytes = est;
            results[idx].reserved_bytes = est;
            used += est;
            fwi_info info;
            if (fwi_model_info(free_slot->model, &info) == FWI_OK)
                results[idx].device_bytes = info.device_bytes;
            ++next;
        }

        bool any_active = false, issued = false;
        for (auto &s : slots) {
            if (s.req < 0) continue;
            any_active = true;
            fwi_result &res = results[s.req];
            if (s.finishing) {
                const cudaError_t q = cudaEventQuery(s.done);
                if (q == cudaErrorNotReady) continue;
                res.t_done = now();
                int rc = q == cudaSuccess ? fwi_sync_status(s.model) : FWI_ERR_CUDA;
                if (q != cudaSuccess) cudaGetLastError();
                const fwi_request &r = reqs[s.req];
                if (rc == FWI_OK) {
                    if (r.kind == FWI_REQ_FORWARD) {
                        if (r.traces_out) std::memcpy(r.traces_out, s.out_pinned, s.out_bytes);
                    } else {
                        if (r.grad_out) std::memcpy(r.grad_out, s.out_pinned, s.out_bytes);
                        res.misfit = *s.misfit_pinned;
                    }
                }
                res.status = rc;
                used -= s.bytes;
                release(s);
                ++finished;
                continue;
            }
            if (s.issued_all || s.pool >= 0) continue;
            // keep at most two turns in flight: skip while the previous turn still runs
            if (cudaEventQuery(s.turn) == cudaErrorNotReady) continue;
            if (res.t_start == 0.0) res.t_start = now();
            bool done = false;
            int rc = fwi::job_advance(s.job, o.steps_per_turn, &done);
            if (rc == FWI_OK && done) {
                rc = fwi::job_finish(s.job, s.misfit_pinned, s.out_pinned);
                s.issued_all = true;
                s.finishing = rc == FWI_OK;
                if (rc == FWI_OK && cudaEventRecord(s.done, s.stream) != cudaSuccess) rc = FWI_ERR_CUDA;
            } else if (rc == FWI_OK && cudaEventRecord(s.turn, s.stream) != cudaSuccess) {
                rc = FWI_ERR_CUDA;
            }
            if (rc != FWI_OK) {
                cudaStreamSynchronize(s.stream);
                res.status = rc;
                res.t_done = now();
                used -= s.bytes;
                release(s);
                ++finished;
                continue;
            }
            issued = true;
        }
        // shared-launch ticks
        for (Pool &pl : pools) {
            if (pl.members.empty()) continue;
            if (pl.pending[pl.buf]) {   // two ticks in flight: wait for the older upload
                if (cudaEventQuery(pl.uploaded[pl.buf]) == cudaErrorNotReady) continue;
                pl.pending[pl.buf] = false;
            }
            fwi::Batch2d *h = pl.host[pl.buf];
            int work = 0, recs = 0, rc = FWI_OK;
            // z-chunk rows per work item: about one item per resident CTA, so a step's
            // critical path (one CTA streaming its chunk) stays short, but no shorter
            // than the 2M warm-up rows each chunk streams
            int64_t row_tiles = 0;
            for (int si : pl.members) {
                const fwi_request &r = reqs[slots[si].req];
                row_tiles += (int64_t)((r.shape[2] + 2 * o.nb + 255) / 256) * (r.shape[0] + 2 * o.nb);
            }
            const int zchunk = (int)std::max<int64_t>(
                2 * pl.M, std::min<int64_t>(kPoolZChunk, (row_tiles + pl.grid_step - 1) / pl.grid_step));
            h->count = 0;
            for (int si : pl.members) {
                Slot &s = slots[si];
                fwi::Batch2dEntry &e = h->e[h->count++];
                rc = fwi::job_batch_entry(s.job, &e, zchunk);
                if (rc != FWI_OK) break;
                e.work0 = work;
                e.rec0 = recs;
                work += e.xtiles * e.p.nzchunks;
                recs += e.nsamp;
                if (!s.pool_synced) {
                    if (cudaStreamWaitEvent(pl.stream, s.turn, 0) != cudaSuccess) rc = FWI_ERR_CUDA;
                    s.pool_synced = true;
                }
                if (results[s.req].t_start == 0.0) results[s.req].t_start = now();
            }
            h->total_work = work;
            h->total_rec = recs;
            const size_t bytes = offsetof(fwi::Batch2d, e) + (size_t)h->count * sizeof(fwi::Batch2dEntry);
            if (pl.kind == 1 && rc == FWI_OK) {
                // one cluster per request, shared memory for the largest band pair
                int64_t need = 0;
                for (int q = 0; q < h->count; ++q) {
                    const fwi::StepParams &sp = h->e[q].p;
                    need = std::max<int64_t>(need, 2LL * ((sp.g.nz + pl.C - 1) / pl.C) * sp.g.px * 4);
                }
                cudaKernelNodeParams kp = pl.params[0];
                kp.gridDim = dim3((unsigned)(pl.C * h->count), 1, 1);
                kp.sharedMemBytes = (unsigned)((need + 1023) / 1024 * 1024);
                if (cudaGraphExecKernelNodeSetParams(pl.exec, pl.nodes[0], &kp) != cudaSuccess) rc = FWI_ERR_CUDA;
            }
            // grids sized to this tick's work (the persistent loops cover any excess)
            const unsigned gs = (unsigned)std::max(1, std::min(work, pl.grid_step));
            const unsigned gr = (unsigned)std::max(1, std::min((recs + 255) / 256, pl.grid_sample));
            // the sampling nodes run only when some request's step does not sample itself
            const bool sample = recs > 0;
            for (size_t q = 0; pl.kind == 0 && rc == FWI_OK && q < pl.nodes.size(); ++q) {
                if ((q & 1) && sample != pl.sampling &&
                    cudaGraphNodeSetEnabled(pl.exec, pl.nodes[q], sample ? 1 : 0) != cudaSuccess)
                    rc = FWI_ERR_CUDA;
                if ((q & 1) && !sample) continue;
                cudaKernelNodeParams kp = pl.params[q];
                kp.gridDim = dim3((q & 1) ? gr : gs, 1, 1);
                if (cudaGraphExecKernelNodeSetParams(pl.exec, pl.nodes[q], &kp) != cudaSuccess) rc = FWI_ERR_CUDA;
            }
            pl.sampling = sample;
            if (rc == FWI_OK && (cudaMemcpyAsync(pl.dev, h, bytes, cudaMemcpyHostToDevice, pl.stream) != cudaSuccess ||
                                 cudaEventRecord(pl.uploaded[pl.buf], pl.stream) != cudaSuccess ||
                                 cudaGraphLaunch(pl.exec, pl.stream) != cudaSuccess))
                rc = FWI_ERR_CUDA;
            if (rc != FWI_OK) {   // the pool's requests fail; the loop goes on
                cudaGetLastError();
                cudaStreamSynchronize(pl.stream);
                for (int si : pl.members) {
                    Slot &s = slots[si];
                    results[s.req].status = rc;
                    results[s.req].t_done = now();
                    used -= s.bytes;
                    release(s);
                    ++finished;
                }
                pl.members.clear();
                continue;
            }
            pl.pending[pl.buf] = true;
            pl.buf ^= 1;
            issued = true;
            // advance the jobs; requests that reached their last step leave the pool
            bool recorded = false;
            std::vector<int> keep;
            for (int si : pl.members) {
                Slot &s = slots[si];
                bool done = false;
                fwi::job_batch_moved(s.job, pl.k, &done);
                if (!done) {
                    keep.push_back(si);
                    continue;
                }
                int frc = FWI_OK;
                if (!recorded) {
                    if (cudaEventRecord(pl.tick, pl.stream) != cudaSuccess) frc = FWI_ERR_CUDA;
                    recorded = true;
                }
                if (frc == FWI_OK && cudaStreamWaitEvent(s.stream, pl.tick, 0) != cudaSuccess) frc = FWI_ERR_CUDA;
                if (frc == FWI_OK) frc = fwi::job_finish(s.job, s.misfit_pinned, s.out_pinned);
                if (frc == FWI_OK && cudaEventRecord(s.done, s.stream) != cudaSuccess) frc = FWI_ERR_CUDA;
                s.pool = -1;
                s.issued_all = true;
                if (frc == FWI_OK) {
                    s.finishing = true;
                } else {
                    cudaGetLastError();
                    cudaStreamSynchronize(s.stream);
                    results[s.req].status = frc;
                    results[s.req].t_done = now();
                    used -= s.bytes;
                    release(s);
                    ++finished;
                }
            }
            pl.members.swap(keep);
        }
        if (!any_active && next < order.size()) {
            // idle until the next arrival
            const double wait = reqs[order[next]].arrival - now();
            if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double>(std::min(wait, 0.01)));
        } else if (!issued) {
            std::this_thread::yield();
        }
    }
    for (Pool &pl : pools) pool_release(pl);
    return FWI_OK;
}
