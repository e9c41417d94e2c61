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
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "fwi.h"

namespace fwi {
struct Job;
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
};

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
            if (s.issued_all) continue;
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
        if (!any_active && next < order.size()) {
            // idle until the next arrival
            const double wait = reqs[order[next]].arrival - now();
            if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double>(std::min(wait, 0.01)));
        } else if (!issued) {
            std::this_thread::yield();
        }
    }
    return FWI_OK;
}
