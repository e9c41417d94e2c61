// C ABI of libfwi (include/fwi.h): model set-up, workspace, and the executors of the
// forward sweep, the checkpointed reverse sweep (gradient) and the source adjoint.
// Every step of the hot path runs in the library's CUDA kernels; this file only
// validates arguments, owns device memory and orders launches on the caller's stream.
#include "fwi.h"

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "fwi_internal.h"
#include "step3d.h"

namespace fwi {
std::vector<int32_t> revolve_actions(int32_t nsteps, int32_t nslots, int64_t *n_forward);
int report_error(int code, const std::string &msg);
}

using namespace fwi;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

}  // namespace

// Sets this thread's error message for entry points defined in other files.
int fwi::report_error(int code, const std::string &msg) { return fail(code, msg); }

namespace {

#define FWI_CU(call)                                                                     \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(e_ == cudaErrorMemoryAllocation ? FWI_ERR_OOM : FWI_ERR_CUDA,    \
                        std::string(#call) + ": " + cudaGetErrorString(e_));             \
    } while (0)

#define FWI_TRY(expr)             \
    do {                          \
        int rc_ = (expr);         \
        if (rc_ != FWI_OK) return rc_; \
    } while (0)

// a kernel launch of the library, counted on the model
#define FWI_LAUNCH(model, call)   \
    do {                          \
        ++(model)->launches;      \
        FWI_CU(call);             \
    } while (0)

// ---------------------------------------------------------------- host numerics

// Central second-derivative weights of radius M (order 2M), the symmetric stencil exact
// on polynomials of degree <= 2M+1:  c_k = 2 (-1)^{k+1} (M!)^2 / (k^2 (M-k)! (M+k)!),
// c_0 = -2 sum_k c_k  (Taylor weights; the paper uses stencils of order >= 8, Sec. 3).
int host_coeffs(int M, double *c)
{
    if (M < 1 || M > kMaxM) return FWI_ERR_ARG;
    double total = 0.0;
    for (int k = 1; k <= M; ++k) {
        // (M!)^2 / ((M-k)! (M+k)!) = prod_{i=1..k} (M - k + i) / (M + i)
        double ratio = 1.0;
        for (int i = 1; i <= k; ++i) ratio *= (double)(M - k + i) / (double)(M + i);
        c[k] = ((k & 1) ? 2.0 : -2.0) * ratio / ((double)k * k);
        total += c[k];
    }
    c[0] = -2.0 * total;
    return FWI_OK;
}

// largest magnitude of the 1-D stencil's symbol (at the Nyquist wavenumber)
double host_symbol_max(int M)
{
    double c[kMaxM + 1] = {};
    if (host_coeffs(M, c) != FWI_OK) return 0.0;   // callers validate M first
    double s = c[0];
    for (int k = 1; k <= M; ++k) s += 2.0 * c[k] * ((k & 1) ? -1.0 : 1.0);
    return std::fabs(s);
}

double host_cfl(int ndim, int M, const float *h, double vmax, double dt)
{
    const double S = host_symbol_max(M);
    double acc = S / ((double)h[0] * h[0]) + S / ((double)h[2] * h[2]);
    if (ndim == 3) acc += S / ((double)h[1] * h[1]);
    return vmax * dt * std::sqrt(acc) / 2.0;
}

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    int ensure(size_t want)
    {
        if (want <= bytes && p) return FWI_OK;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        if (want == 0) return FWI_OK;
        cudaError_t e = cudaMalloc(&p, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return fail(FWI_ERR_OOM, "cudaMalloc of " + std::to_string(want) + " bytes failed");
        }
        bytes = want;
        return FWI_OK;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <class T> T *as() const { return (T *)p; }
};

int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

}  // namespace

struct fwi_model {
    int ndim = 0, M = 0, order = 0, nb = 0, nt = 0;
    int64_t np[3] = {0, 0, 0};
    float h[3] = {0, 0, 0};
    float dt = 0;
    fwi_opts opts{};
    Geom g{};
    Coefs co{};
    float vmax = 0, vref = 0, cfl = 0, eta_max[3] = {0, 0, 0};
    // model
    DevBuf v, W, sig;   // sig: sig_z[nz] | sig_y[ny] | sig_x[nx]
    // workspace
    int cap_shots = 0, cap_nrec = 0;
    DevBuf u[2], mu[2], g32, g64, traces, src_off, rec_off, inj, src_scale, maxbits, partials,
        phi, snaps, scales, src_pts, rec_pts, step_ctr, ut[2];   // ut: spare forward states
    DevBuf stage_in[3], stage_out[2];
    int nslots = 0;
    size_t slot_bytes = 0;
    // cached geometry (nodes, or positions of off-grid points)
    std::vector<int32_t> geo_src, geo_rec;
    std::vector<double> geo_src_pos, geo_rec_pos;
    int geo_shots = -1, geo_nrec = -1;
    bool og_src = false, og_rec = false;   // current acquisition uses off-grid points
    // cached schedule
    int sched_nslots = -1, sched_nt = -1;
    int sched_npair = 0;               // slots that ever hold a pair
    std::vector<int64_t> slot_off;     // slot k starts slot_off[k] half slots into the pool
    std::vector<char> slot_pair;       // slot k holds pairs (two fields per shot)
    int64_t snaps_layout = -1;   // code layout the pool was last zeroed for
    std::vector<int32_t> sched;
    std::vector<int> sched_comps;   // per action: checkpoint components moved (1 or 2)
    int64_t sched_fwd = 0;
    // status
    unsigned *h_flag = nullptr, *d_flag = nullptr;
    cudaStream_t last_stream = nullptr;
    // stats of the last gradient call
    int64_t st_fwd = 0, st_adj = 0, st_store = 0, st_restore = 0;
    // launch count and kernel timing (opts.timing)
    int64_t launches = 0;
    std::vector<cudaEvent_t> ev;
    std::vector<int> ev_kind;   // per event pair: 0 forward step, 1 reverse step, 2 forward
                                // step that also writes a checkpoint
    size_t ev_used = 0;
    // TMA tensor maps of the 3-D step, keyed by buffer, shot count and box
    struct MapEntry {
        const void *base;
        int ns, bx, by, eb;
        int64_t stride;
        CUtensorMap map;
    };
    std::vector<MapEntry> maps;
    std::vector<MapEntry> maps2;   // 3-D maps of 2-D fields
    // 3-D: every receiver a node of computed plane rec_fuse_z, distinct per shot: the step
    // kernels sample and inject at them from rec_map ([shot][y][x] receiver index or -1);
    // -1 otherwise
    DevBuf rec_map;
    int rec_fuse_z = -1;
    DevBuf cl_tab;                 // one-entry table of the on-chip 2-D forward launch
    Batch2d *cl_host = nullptr;    // its pinned staging
    cudaEvent_t cl_up = nullptr;   // the staging's last upload finished
    int cl_rec_z = -1, cl_rec_x0 = 0;
    int resident[3] = {0, 0, 0};   // resident CTAs of the 3-D step kernel, per mode
    int resident_query[3] = {0, 0, 0};   // what the occupancy query returned (-e: error e)
    int64_t t_fwd_n = 0, t_adj_n = 0, t_st_n = 0;
    double t_fwd_ms = 0.0, t_adj_ms = 0.0, t_st_ms = 0.0;

    int64_t device_bytes() const
    {
        size_t b = v.bytes + W.bytes + sig.bytes + g32.bytes + g64.bytes + traces.bytes +
                   src_off.bytes + rec_off.bytes + inj.bytes + src_scale.bytes + maxbits.bytes +
                   partials.bytes + phi.bytes + snaps.bytes + scales.bytes + rec_map.bytes;
        for (int i = 0; i < 2; ++i) b += u[i].bytes + mu[i].bytes + stage_out[i].bytes;
        for (int i = 0; i < 3; ++i) b += stage_in[i].bytes;
        return (int64_t)b;
    }
};

namespace {

const float *sig_z(const fwi_model *m) { return m->sig.as<float>(); }
const float *sig_y(const fwi_model *m) { return m->sig.as<float>() + m->g.nz; }
const float *sig_x(const fwi_model *m) { return m->sig.as<float>() + m->g.nz + m->g.ny; }

int check_status(fwi_model *m)
{
    const unsigned st = m->h_flag ? *(volatile unsigned *)m->h_flag : 0u;
    if (st & 2u)
        return fail(FWI_ERR_TIMEOUT, "a bounded device wait ran out (latched device status)");
    if (st & 1u)
        return fail(FWI_ERR_UNSTABLE, "a wavefield became non-finite (latched device status)");
    return FWI_OK;
}

// Copies a caller input (host or device) to the device; returns a device pointer.
int stage_input(fwi_model *m, int slot, const void *src, size_t bytes, cudaStream_t s,
                const void **dev)
{
    if (is_device_ptr(src)) {
        *dev = src;
        return FWI_OK;
    }
    FWI_TRY(m->stage_in[slot].ensure(bytes));
    FWI_CU(cudaMemcpyAsync(m->stage_in[slot].p, src, bytes, cudaMemcpyHostToDevice, s));
    *dev = m->stage_in[slot].p;
    return FWI_OK;
}

// Device pointer an output can be written to: the caller's (device) or a staging buffer.
int output_target(fwi_model *m, int slot, void *dst, size_t bytes, void **dev, bool *host)
{
    *host = !is_device_ptr(dst);
    if (!*host) {
        *dev = dst;
        return FWI_OK;
    }
    FWI_TRY(m->stage_out[slot].ensure(bytes));
    *dev = m->stage_out[slot].p;
    return FWI_OK;
}

// Velocity-dependent state: copy v, largest velocity, sponge tables, CFL check, W.
int set_velocity(fwi_model *m, const float *vp, cudaStream_t s)
{
    const int64_t nphys = m->np[0] * m->np[1] * m->np[2];
    FWI_TRY(m->v.ensure(nphys * sizeof(float)));
    FWI_CU(cudaMemcpyAsync(m->v.p, vp, nphys * sizeof(float), cudaMemcpyDefault, s));
    // largest velocity through the codec's max|.| kernel (v > 0)
    FWI_TRY(m->maxbits.ensure(128 * sizeof(unsigned)));
    FWI_CU(cudaMemsetAsync(m->maxbits.p, 0, 2 * sizeof(unsigned), s));
    FWI_LAUNCH(m, launch_maxabs(m->v.as<float>(), m->v.as<float>(), nphys, nphys, 1,
                         m->maxbits.as<unsigned>(), s));
    unsigned bits = 0;
    FWI_CU(cudaMemcpyAsync(&bits, m->maxbits.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    FWI_CU(cudaStreamSynchronize(s));
    float vmax;
    std::memcpy(&vmax, &bits, sizeof(float));
    if (!(vmax > 0.0f) || !std::isfinite(vmax))
        return fail(FWI_ERR_ARG, "velocity must be finite and positive");
    m->vmax = vmax;
    m->vref = m->opts.sponge_vref > 0.0f ? m->opts.sponge_vref : vmax;
    m->cfl = (float)host_cfl(m->ndim, m->M, m->h, vmax, m->dt);
    if (!(m->cfl < 1.0f)) {
        char buf[160];
        std::snprintf(buf, sizeof buf,
                      "dt = %g s violates the stability limit: v_max dt sqrt(sum S/h^2)/2 = %g >= 1",
                      (double)m->dt, (double)m->cfl);
        return fail(FWI_ERR_CFL, buf);
    }
    // sponge: eta_a(i) = eta_max,a (depth_a(i)/nb)^2, eta_max,a = 3 vref ln(1/R0)/(2 nb h_a);
    // the kernels read s = eta dt / 2 per axis
    const int nb = m->nb;
    const int ext[3] = {m->g.nz, m->g.ny, m->g.nx};
    // 4 floats of padding: the 3-D step copies sig_z in 16-byte aligned groups of four
    std::vector<float> sig(ext[0] + ext[1] + ext[2] + 4, 0.0f);
    size_t base = 0;
    for (int a = 0; a < 3; ++a) {
        const bool present = !(a == 1 && m->ndim == 2);
        double emax = 0.0;
        if (present && nb > 0)
            emax = 3.0 * m->vref * std::log(1.0 / m->opts.sponge_r0) / (2.0 * nb * m->h[a]);
        m->eta_max[a] = (float)emax;
        for (int i = 0; i < ext[a]; ++i) {
            double d = 0.0;
            if (present && nb > 0) {
                if (i < nb) d = nb - i;
                else if (i >= nb + m->np[a]) d = i - (nb + m->np[a] - 1);
            }
            const double eta = emax * (d / nb) * (d / nb);
            sig[base + i] = (float)(0.5 * m->dt * (nb > 0 ? eta : 0.0));
        }
        base += ext[a];
    }
    FWI_TRY(m->sig.ensure(sig.size() * sizeof(float)));
    FWI_CU(cudaMemcpyAsync(m->sig.p, sig.data(), sig.size() * sizeof(float),
                           cudaMemcpyHostToDevice, s));
    FWI_TRY(m->W.ensure(m->g.field * sizeof(float)));
    FWI_CU(cudaMemsetAsync(m->W.p, 0, m->g.field * sizeof(float), s));
    FWI_LAUNCH(m, launch_build_W(m->g, nb, m->np, m->v.as<float>(), m->dt, m->W.as<float>(), s));
    FWI_CU(cudaStreamSynchronize(s));   // `sig` is a host temporary
    return FWI_OK;
}

// Kaiser-windowed sinc weights of an off-grid point along one axis (Hicks 2002,
// Geophysics 67(1)): the 8 nodes first .. first + 7 around the computed-grid coordinate p
// get sinc(x - p) I0(6.31 sqrt(1 - ((x - p) / 4)^2)) / I0(6.31).  At integer p the weights
// are the delta at p.
void sinc_weights(double p, int32_t *first, float *w)
{
    auto i0 = [](double x) {   // modified Bessel function of order 0, power series
        double term = 1.0, total = 1.0;
        const double q = x * x / 4.0;
        for (int k = 1; k < 400 && term > 1e-18 * total; ++k) {
            term = term * q / ((double)k * k);
            total += term;
        }
        return total;
    };
    const double kb = 6.31, half = kTaps / 2, pi = 3.14159265358979323846;
    const double fl = std::floor(p);
    *first = (int32_t)fl - (int32_t)half + 1;
    const double norm = i0(kb);
    for (int k = 0; k < kTaps; ++k) {
        const double t = (double)(*first + k) - p;
        double sinc;
        if (t == std::floor(t)) sinc = (t == 0.0) ? 1.0 : 0.0;
        else sinc = std::sin(pi * t) / (pi * t);
        const double r = t / half;
        const double win = (r >= -1.0 && r <= 1.0) ? i0(kb * std::sqrt(1.0 - r * r)) / norm : 0.0;
        w[k] = (float)(sinc * win);
    }
}

// Taps of the off-grid point at physical-grid position pos (z, y, x); false when a tap
// would fall outside the computed grid.
bool point_taps(const fwi_model *m, const double *pos, PointTaps *out)
{
    const int nby = m->ndim == 3 ? m->nb : 0;
    const double c[3] = {pos[0] + m->nb, pos[1] + nby, pos[2] + m->nb};
    const int64_t n[3] = {m->g.nz, m->g.ny, m->g.nx};
    int32_t first[3] = {0, 0, 0};
    for (int a = 0; a < 3; ++a) {
        if (a == 1 && m->ndim == 2) {
            out->w[kTaps] = 1.0f;
            for (int k = 1; k < kTaps; ++k) out->w[kTaps + k] = 0.0f;
            continue;
        }
        sinc_weights(c[a], &first[a], out->w + a * kTaps);
        if (first[a] < 0 || first[a] + kTaps > n[a]) return false;
    }
    out->z0 = first[0];
    out->y0 = first[1];
    out->x0 = first[2];
    out->pad = 0;
    return true;
}

int validate_acq(const fwi_model *m, const fwi_acq *a)
{
    if (!a || a->nshots < 1 || a->nrec < 1 || (!a->src && !a->src_pos) ||
        (!a->rec && !a->rec_pos))
        return fail(FWI_ERR_ARG, "acquisition needs nshots >= 1, nrec >= 1, sources and "
                                 "receivers (nodes or positions)");
    if ((int64_t)a->nshots * 65535 < a->nshots)
        return fail(FWI_ERR_ARG, "too many shots");
    auto inside_pos = [&](const double *p) {
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(p[k])) return false;
        if (!(p[0] >= 0.0 && p[0] <= (double)(m->np[0] - 1) && p[2] >= 0.0 &&
              p[2] <= (double)(m->np[2] - 1)))
            return false;
        if (m->ndim == 3) return p[1] >= 0.0 && p[1] <= (double)(m->np[1] - 1);
        return p[1] == 0.0;
    };
    PointTaps t;
    if (a->src_pos)
        for (int s = 0; s < a->nshots; ++s)
            if (!inside_pos(a->src_pos + 3 * s) || !point_taps(m, a->src_pos + 3 * s, &t))
                return fail(FWI_ERR_ARG, "source position " + std::to_string(s) +
                                             " outside the grid or its taps outside the "
                                             "sponge (nb >= 4 needed near the edges)");
    if (a->rec_pos)
        for (int64_t i = 0; i < (int64_t)a->nshots * a->nrec; ++i)
            if (!inside_pos(a->rec_pos + 3 * i) || !point_taps(m, a->rec_pos + 3 * i, &t))
                return fail(FWI_ERR_ARG, "receiver position " + std::to_string(i) +
                                             " outside the grid or its taps outside the "
                                             "sponge (nb >= 4 needed near the edges)");
    auto inside = [&](const int32_t *p) {
        if (p[0] < 0 || p[0] >= m->np[0] || p[2] < 0 || p[2] >= m->np[2]) return false;
        if (m->ndim == 3) return p[1] >= 0 && p[1] < m->np[1];
        return p[1] == 0;
    };
    for (int s = 0; s < a->nshots; ++s) {
        if (!a->src_pos && !inside(a->src + 3 * s))
            return fail(FWI_ERR_ARG, "source " + std::to_string(s) + " outside the grid");
        for (int r = 0; r < a->nrec && !a->rec_pos; ++r)
            if (!inside(a->rec + 3 * ((int64_t)s * a->nrec + r)))
                return fail(FWI_ERR_ARG, "receiver " + std::to_string(r) + " of shot " +
                                             std::to_string(s) + " outside the grid");
    }
    return FWI_OK;
}

int64_t node_offset(const fwi_model *m, const int32_t *p)
{
    const int nby = m->ndim == 3 ? m->nb : 0;
    return (int64_t)(p[0] + m->nb) * m->g.plane + (int64_t)(p[1] + nby) * m->g.px + (p[2] + m->nb);
}

// Per-shot buffers for `nshots` shots and `nrec` receivers; `grad` adds the reverse-sweep
// fields.  Uploads the source/receiver offsets when the geometry changed.
int ensure_workspace(fwi_model *m, const fwi_acq *a, bool grad, cudaStream_t s)
{
    const int ns = a->nshots, nr = a->nrec;
    const size_t fb = (size_t)m->g.field * sizeof(float);
    FWI_TRY(m->u[0].ensure(ns * fb));
    FWI_TRY(m->u[1].ensure(ns * fb));
    FWI_TRY(m->traces.ensure((size_t)ns * m->nt * nr * sizeof(float)));
    FWI_TRY(m->src_off.ensure(ns * sizeof(int64_t)));
    FWI_TRY(m->rec_off.ensure((size_t)ns * nr * sizeof(int64_t)));
    FWI_TRY(m->inj.ensure((size_t)ns * nr * sizeof(float)));
    FWI_TRY(m->src_scale.ensure(ns * sizeof(float)));
    FWI_TRY(m->maxbits.ensure(2 * (ns > 64 ? ns : 64) * sizeof(unsigned)));
    FWI_TRY(m->partials.ensure(1024 * sizeof(double)));
    FWI_TRY(m->phi.ensure(sizeof(double)));
    if (grad) {
        FWI_TRY(m->mu[0].ensure(ns * fb));
        FWI_TRY(m->mu[1].ensure(ns * fb));
        FWI_TRY(m->g32.ensure(ns * fb));
        FWI_TRY(m->g64.ensure(ns * 2 * fb));
    }
    if (ns > m->cap_shots) m->cap_shots = ns;
    if (nr > m->cap_nrec) m->cap_nrec = nr;
    const size_t nsrc = (size_t)ns * 3, nrec3 = (size_t)ns * nr * 3;
    auto same_i = [](const std::vector<int32_t> &v, const int32_t *p, size_t n) {
        return p ? (v.size() == n && std::memcmp(v.data(), p, n * sizeof(int32_t)) == 0)
                 : v.empty();
    };
    auto same_d = [](const std::vector<double> &v, const double *p, size_t n) {
        return p ? (v.size() == n && std::memcmp(v.data(), p, n * sizeof(double)) == 0)
                 : v.empty();
    };
    const bool og_s = a->src_pos != nullptr, og_r = a->rec_pos != nullptr;
    bool same = m->geo_shots == ns && m->geo_nrec == nr &&
                (og_s ? same_d(m->geo_src_pos, a->src_pos, nsrc) : same_i(m->geo_src, a->src, nsrc)) &&
                (og_r ? same_d(m->geo_rec_pos, a->rec_pos, nrec3) : same_i(m->geo_rec, a->rec, nrec3)) &&
                m->og_src == og_s && m->og_rec == og_r;
    if (!same) {
        std::vector<int64_t> so(ns, 0), ro((size_t)ns * nr, 0);
        std::vector<PointTaps> sp, rp;
        if (og_s) {
            sp.resize(ns);
            for (int i = 0; i < ns; ++i) point_taps(m, a->src_pos + 3 * i, &sp[i]);
            FWI_TRY(m->src_pts.ensure(sp.size() * sizeof(PointTaps)));
        } else {
            for (int i = 0; i < ns; ++i) so[i] = node_offset(m, a->src + 3 * i);
        }
        if (og_r) {
            rp.resize((size_t)ns * nr);
            for (size_t i = 0; i < rp.size(); ++i) point_taps(m, a->rec_pos + 3 * i, &rp[i]);
            FWI_TRY(m->rec_pts.ensure(rp.size() * sizeof(PointTaps)));
        } else {
            for (size_t i = 0; i < (size_t)ns * nr; ++i) ro[i] = node_offset(m, a->rec + 3 * i);
        }
        FWI_CU(cudaMemcpyAsync(m->src_off.p, so.data(), ns * sizeof(int64_t),
                               cudaMemcpyHostToDevice, s));
        FWI_CU(cudaMemcpyAsync(m->rec_off.p, ro.data(), ro.size() * sizeof(int64_t),
                               cudaMemcpyHostToDevice, s));
        if (og_s)
            FWI_CU(cudaMemcpyAsync(m->src_pts.p, sp.data(), sp.size() * sizeof(PointTaps),
                                   cudaMemcpyHostToDevice, s));
        if (og_r)
            FWI_CU(cudaMemcpyAsync(m->rec_pts.p, rp.data(), rp.size() * sizeof(PointTaps),
                                   cudaMemcpyHostToDevice, s));
        // receivers on one plane at distinct nodes: map them for the step kernels
        m->rec_fuse_z = -1;
        std::vector<int32_t> rmap;
        const char *fz = std::getenv("FWI_STEP3D_REC_FUSE");   // 0: separate kernels
        if (m->ndim == 3 && !og_r && nr > 0 && !(fz && std::atoi(fz) == 0)) {
            const int64_t plane = m->g.plane;
            const int z0 = (int)(ro[0] / plane);
            bool ok = true;
            for (size_t i = 0; ok && i < ro.size(); ++i) ok = ro[i] / plane == z0;
            if (ok) {
                rmap.assign((size_t)ns * plane, -1);
                for (int sh = 0; ok && sh < ns; ++sh)
                    for (int r = 0; ok && r < nr; ++r) {
                        int32_t &slot = rmap[(size_t)sh * plane + (size_t)(ro[(size_t)sh * nr + r] % plane)];
                        ok = slot < 0;
                        slot = r;
                    }
            }
            if (ok && m->rec_map.ensure(rmap.size() * sizeof(int32_t)) == FWI_OK) {
                FWI_CU(cudaMemcpyAsync(m->rec_map.p, rmap.data(), rmap.size() * sizeof(int32_t),
                                       cudaMemcpyHostToDevice, s));
                m->rec_fuse_z = z0;
            }
        }
        FWI_CU(cudaStreamSynchronize(s));   // host temporaries
        if (og_s) { m->geo_src.clear(); m->geo_src_pos.assign(a->src_pos, a->src_pos + nsrc); }
        else { m->geo_src_pos.clear(); m->geo_src.assign(a->src, a->src + nsrc); }
        if (og_r) { m->geo_rec.clear(); m->geo_rec_pos.assign(a->rec_pos, a->rec_pos + nrec3); }
        else { m->geo_rec_pos.clear(); m->geo_rec.assign(a->rec, a->rec + nrec3); }
        m->geo_shots = ns;
        m->geo_nrec = nr;
        m->og_src = og_s;
        m->og_rec = og_r;
    }
    return FWI_OK;
}

StepParams base_params(const fwi_model *m)
{
    StepParams p{};
    p.g = m->g;
    p.c = m->co;
    p.W = m->W.as<float>();
    p.sig_z = sig_z(m);
    p.sig_y = sig_y(m);
    p.sig_x = sig_x(m);
    p.nt = m->nt;
    p.dt2 = m->dt * m->dt;
    return p;
}

// One time-step launch (kind 0: forward, 1: reverse); bracketed by CUDA events on the
// launching stream when timing is on.
// Tensor map of `ns` shots of a field (elements of eb bytes, shots `stride` elements
// apart; stride 0 = the field layout), cached per model.
int field_map(fwi_model *m, const void *base, int ns, int bx, int by, CUtensorMap *out,
              int eb = 4, int64_t stride = 0)
{
    if (stride == 0) stride = m->g.field;
    for (const auto &e : m->maps)
        if (e.base == base && e.ns == ns && e.bx == bx && e.by == by && e.eb == eb &&
            e.stride == stride) {
            *out = e.map;
            return FWI_OK;
        }
    fwi_model::MapEntry e{base, ns, bx, by, eb, stride, {}};
    if (encode_field_map(&e.map, base, m->g, ns, bx, by, eb, stride) != 0)
        return fail(FWI_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    m->maps.push_back(e);
    *out = e.map;
    return FWI_OK;
}

// Resident CTAs of each 3-D step mode, queried once per model (outside any capture).
void ensure_resident(fwi_model *m)
{
    const bool iso = m->h[0] == m->h[1] && m->h[1] == m->h[2];
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        sms = 152;
    }
    for (int mode = 0; mode < 3; ++mode)
        if (m->resident[mode] <= 0) {
            const int r = step3d_resident_ctas(m->g.M, mode, iso);
            m->resident_query[mode] = r;
            m->resident[mode] = r > 0 ? r : sms;   // one CTA per SM if the query failed
            // tuning runs: FWI_STEP3D_PER_SM=<k> plans k CTAs per SM instead
            if (const char *e = std::getenv("FWI_STEP3D_PER_SM"))
                if (std::atoi(e) > 0) m->resident[mode] = sms * std::atoi(e);
        }
}

// One launch of the TMA-staged 3-D kernel (k_step3d.cu) in `mode`.
int step3d_launch(fwi_model *m, const StepParams &p, int ns, int mode, cudaStream_t s)
{
    const Geom &g = m->g;
    Step3dParams q{};
    q.M = g.M;
    q.nx = g.nx;
    q.ny = g.ny;
    q.nz = g.nz;
    q.px = g.px;
    q.plane = g.plane;
    q.field = g.field;
    for (int k = 0; k <= kMaxM; ++k) {
        q.cx[k] = m->co.cx[k];
        q.cy[k] = m->co.cy[k];
        q.cz[k] = m->co.cz[k];
        q.cy2[k] = make_float2(m->co.cy[k], m->co.cy[k]);
        q.cz2[k] = make_float2(m->co.cz[k], m->co.cz[k]);
    }
    q.c0 = m->co.c0;
    q.c02 = make_float2(m->co.c0, m->co.c0);
    q.iso = m->h[0] == m->h[1] && m->h[1] == m->h[2];
    q.inv_h2 = (float)(1.0 / ((double)m->h[0] * m->h[0]));
    q.sig_x = sig_x(m);
    q.sig_y = sig_y(m);
    q.sig_z = sig_z(m);
    q.err = m->d_flag;
    if (mode == kModeStep && p.st_code) mode = kModeStepStore;
    const int TY = step3d_variant(g.M, mode).ty;
    CUtensorMap mc, ma, mb, md, me;
    FWI_TRY(field_map(m, p.cur, ns, 64 + 2 * g.M, TY + 2 * g.M, &mc));
    FWI_TRY(field_map(m, p.prev, ns, 64, TY, &ma));
    FWI_TRY(field_map(m, m->W.p, 1, 64, TY, &mb));
    q.out = p.prev;
    q.src_off = p.src_off;
    q.wavelet = p.wavelet;
    q.nt = p.nt;
    q.n = p.n;
    q.n_dev = p.n_dev;
    q.dt2 = p.dt2;
    if (mode == kModeStep && p.st_code) mode = kModeStepStore;
    if (mode == kModeStep || mode == kModeStepStore) {
        q.maxbits = p.maxbits;
        q.st_code = p.st_code;
        q.st_scale = p.st_scale;
        q.st_dtype = p.st_dtype;
        q.st_comps = p.st_comps;
        q.st_cstride = p.st_cstride;
        md = ma;
        me = ma;
    } else {
        FWI_TRY(field_map(m, p.aux, ns, 64, TY, &md, p.aux_fmt ? 2 : 4, p.aux_stride));
        FWI_TRY(field_map(m, p.gacc, ns, 64, TY, &me));
        q.g = p.gacc;
        q.aux_fmt = p.aux_fmt;
        q.aux_scale = p.aux_scale;
    }
    // receivers handled in the epilogue: samples of a forward step that records traces
    // (node source: off-grid source taps are added after the step, before sampling), the
    // residual injection of a reverse step with imaging
    if (m->rec_fuse_z >= 0 &&
        (mode == kModeAdj ? p.inj_q != nullptr : (p.rec_tr != nullptr && !m->og_src))) {
        q.rec_map = m->rec_map.as<int>();
        q.rec_z = m->rec_fuse_z;
        q.nrec = m->geo_nrec;
        q.rec_tr = p.rec_tr;
        q.inj_q = p.inj_q;
        q.inj_scale = p.inj_scale;
        q.inj_n = p.inj_n;
    }
    ensure_resident(m);
    const int tiles = ((g.nx + 63) / 64) * ((g.ny + TY - 1) / TY);
    q.nshots = ns;
    // z-parts in step when the streamed field is larger than the L2 (~126 MB)
    const bool in_step = (double)g.field * 4.0 * ns > 96.0 * (1 << 20);
    const int ctas = plan_persistent(q, tiles * ns, m->resident[mode], in_step);
    FWI_CU(launch_step3d_tma(q, mode, ctas, mc, ma, mb, md, me, s));
    return FWI_OK;
}

bool use_step3d(const fwi_model *m) { return m->ndim == 3; }

// 3-D map [shot][z][x] of a 2-D field, cached per model like field_map's.
int field_map2d(fwi_model *m, const void *base, int ns, int bx, CUtensorMap *out, int eb = 4,
                int64_t stride = 0)
{
    if (stride == 0) stride = m->g.field;
    for (const auto &e : m->maps2)
        if (e.base == base && e.ns == ns && e.bx == bx && e.eb == eb && e.stride == stride) {
            *out = e.map;
            return FWI_OK;
        }
    fwi_model::MapEntry e{base, ns, bx, 1, eb, stride, {}};
    if (encode_field_map2d(&e.map, base, m->g, ns, bx, eb, stride) != 0)
        return fail(FWI_ERR_CUDA, "cuTensorMapEncodeTiled failed (2-D)");
    m->maps2.push_back(e);
    *out = e.map;
    return FWI_OK;
}

// The 2-D step with TMA-staged rows, opt-in (FWI_STEP2D_TMA=1; same results bit for bit
// as the register-streaming kernel).  Measured on GB300, 64 shots of 440 x 1064: forward
// 0.144 against 0.103 ms, forward + store 0.150 against 0.109, reverse 0.157 against
// 0.158 ms.  A 2-D row is 256 points per CTA: per row the staged kernel pays a CTA
// barrier, two mbarrier round trips and five small copies (1 KB and two 16-byte halo
// boxes), which cost more than the L1-served loads they replace; the latency they hide
// in the reverse step only breaks even.
bool use_step2d_tma()
{
    const char *e = std::getenv("FWI_STEP2D_TMA");
    return e && std::atoi(e) != 0;
}

int step2d_tma_launch(fwi_model *m, const StepParams &p, int ns, bool img, cudaStream_t s)
{
    CUtensorMap maps[6];
    FWI_TRY(field_map2d(m, p.cur, ns, 256, &maps[0]));
    FWI_TRY(field_map2d(m, p.cur, ns, m->g.M, &maps[1]));
    FWI_TRY(field_map2d(m, p.prev, ns, 256, &maps[2]));
    FWI_TRY(field_map2d(m, m->W.p, 1, 256, &maps[3]));
    if (img) {
        FWI_TRY(field_map2d(m, p.aux, ns, 256, &maps[4], p.aux_fmt ? 2 : 4, p.aux_stride));
        FWI_TRY(field_map2d(m, p.gacc, ns, 256, &maps[5]));
    } else {
        maps[4] = maps[5] = maps[2];
    }
    StepParams q = p;
    q.err = m->d_flag;
    FWI_CU(launch_step2d_tma(q, ns, img, maps, s));
    return FWI_OK;
}

// The time step itself: in 2-D the register-streaming (or, opt-in, the TMA-staged)
// kernel, in 3-D the TMA kernels; with `img` the reverse step that also accumulates the
// imaging condition.
int raw_step(fwi_model *m, const StepParams &p, int ns, bool img, cudaStream_t s)
{
    if (!use_step3d(m)) {
        if (use_step2d_tma()) return step2d_tma_launch(m, p, ns, img, s);
        FWI_CU(launch_step2d(p, ns, img, s));
        return FWI_OK;
    }
    return step3d_launch(m, p, ns, img ? kModeAdj : kModeStep, s);
}

int step_launch(fwi_model *m, const StepParams &p, int ns, bool img, int kind, cudaStream_t s)
{
    ++m->launches;
    if (!m->opts.timing) return raw_step(m, p, ns, img, s);
    if (m->ev_used + 2 > m->ev.size()) {
        for (int i = 0; i < 256; ++i) {
            cudaEvent_t e;
            FWI_CU(cudaEventCreate(&e));
            m->ev.push_back(e);
        }
    }
    FWI_CU(cudaEventRecord(m->ev[m->ev_used], s));
    FWI_TRY(raw_step(m, p, ns, img, s));
    FWI_CU(cudaEventRecord(m->ev[m->ev_used + 1], s));
    m->ev_used += 2;
    m->ev_kind.push_back(kind);
    return FWI_OK;
}

// Waits for the recorded events and adds their durations to the model's totals.
int collect_timing(fwi_model *m)
{
    if (!m->opts.timing || m->ev_used == 0) return FWI_OK;
    FWI_CU(cudaEventSynchronize(m->ev[m->ev_used - 1]));
    for (size_t i = 0; i < m->ev_kind.size(); ++i) {
        float ms = 0.0f;
        FWI_CU(cudaEventElapsedTime(&ms, m->ev[2 * i], m->ev[2 * i + 1]));
        if (m->ev_kind[i] == 0) {
            m->t_fwd_ms += ms;
            ++m->t_fwd_n;
        } else if (m->ev_kind[i] == 2) {
            m->t_st_ms += ms;
            ++m->t_st_n;
        } else {
            m->t_adj_ms += ms;
            ++m->t_adj_n;
        }
    }
    m->ev_used = 0;
    m->ev_kind.clear();
    return FWI_OK;
}

int set_coefs(fwi_model *m)
{
    double c[kMaxM + 1];
    FWI_TRY(host_coeffs(m->M, c));
    const double iz = 1.0 / ((double)m->h[0] * m->h[0]);
    const double iy = m->ndim == 3 ? 1.0 / ((double)m->h[1] * m->h[1]) : 0.0;
    const double ix = 1.0 / ((double)m->h[2] * m->h[2]);
    for (int k = 0; k <= kMaxM; ++k) {
        const double ck = k <= m->M ? c[k] : 0.0;
        m->co.cz[k] = (float)(ck * iz);
        m->co.cy[k] = (float)(ck * iy);
        m->co.cx[k] = (float)(ck * ix);
    }
    m->co.c0 = (float)(c[0] * (iz + iy + ix));
    return FWI_OK;
}

int finish_output(void *user, const void *dev, size_t bytes, bool host, cudaStream_t s)
{
    if (!user || !host) return FWI_OK;
    FWI_CU(cudaMemcpyAsync(user, dev, bytes, cudaMemcpyDeviceToHost, s));
    return FWI_OK;
}

}  // namespace

// ---------------------------------------------------------------- resumable executors
//
// A forward or gradient evaluation is a job: set-up, then advance() issues the next
// `units` time steps' worth of launches on the job's stream (a unit is one forward or one
// reverse step; checkpoint stores and restores ride along with the step they precede),
// then finish() issues the result copies.  The C ABI runs a job to the end in one call;
// the serving loop interleaves the jobs of many requests on their own streams.

namespace fwi {

struct FwdJob {
    fwi_model *m = nullptr;
    cudaStream_t s = nullptr;
    int ns = 0, nr = 0;
    StepParams p{};
    float *tr = nullptr;    // device traces target (may be null)
    float *uc = nullptr, *up = nullptr;   // u^n and u^{n-1}
    int n = 0;
    int tb_chunks = 0;      // z-chunks of the two-step pass (0: single steps only)
    int cl_size = 0;        // temporal blocking on chip: cluster size (0: off)
    // CUDA graph of one turn: g_units steps from the state buffers (g_uc, g_up), replayed
    // with the device step counter m->step_ctr (dev_n: its value as the host last set it)
    cudaGraphExec_t gexec = nullptr;
    const float *g_uc = nullptr;
    int g_units = 0, dev_n = -1;
    int64_t g_kernels = 0;
    bool g_failed = false;
    FwdJob() = default;
    FwdJob(const FwdJob &) = delete;
    FwdJob &operator=(const FwdJob &) = delete;
    ~FwdJob()
    {
        if (gexec) cudaGraphExecDestroy(gexec);
    }
};

int fwd_setup(FwdJob &j, fwi_model *m, int ns, int nr, const float *wav, float *tr,
              cudaStream_t s)
{
    j.m = m;
    j.s = s;
    j.ns = ns;
    j.nr = nr;
    j.tr = tr;
    const size_t fb = (size_t)m->g.field * sizeof(float);
    FWI_CU(cudaMemsetAsync(m->u[0].p, 0, ns * fb, s));
    FWI_CU(cudaMemsetAsync(m->u[1].p, 0, ns * fb, s));
    j.p = base_params(m);
    // an on-grid source is injected inside the step; off-grid taps right after it
    j.p.src_off = m->og_src ? nullptr : m->src_off.as<int64_t>();
    j.p.wavelet = wav;
    j.uc = m->u[0].as<float>();
    j.up = m->u[1].as<float>();
    j.n = 0;
    // 2-D batches wide enough to fill the GPU advance two steps per pass when the source
    // is a node (off-grid source taps are added between steps)
    j.tb_chunks = (m->og_src || m->opts.temporal_blocking != 1) ? 0 : step2d_tb2_chunks(m->g, ns);
    j.cl_size = 0;
    if (m->opts.temporal_blocking == 2 && m->ndim == 2 && ns == 1 && !m->og_src && !m->og_rec &&
        tr && !m->opts.timing) {
        // receivers on one row (sampled in the step's epilogue) and states that fit on chip
        const int C = cluster2d_size(m->M);
        bool ok = C > 0 && nr > 0 && m->g.nz / C > m->M &&
                  2LL * ((m->g.nz + C - 1) / C) * m->g.px * 4 <= cluster2d_max_smem();
        int64_t o0 = 0;
        if (ok) {
            o0 = node_offset(m, m->geo_rec.data());
            const int x0 = (int)(o0 % m->g.plane);
            ok = x0 + nr <= m->g.nx;
            for (int r = 1; ok && r < nr; ++r) ok = node_offset(m, m->geo_rec.data() + 3 * r) == o0 + r;
        }
        if (ok && m->cl_tab.ensure(sizeof(Batch2d)) == FWI_OK) {
            if (!m->cl_host) {
                if (cudaMallocHost((void **)&m->cl_host, sizeof(Batch2d)) != cudaSuccess) {
                    cudaGetLastError();
                    m->cl_host = nullptr;
                }
            }
            if (m->cl_host) {
                j.cl_size = C;
                m->cl_rec_z = (int)(o0 / m->g.plane);
                m->cl_rec_x0 = (int)(o0 % m->g.plane);
            }
        }
    }
    if (j.tb_chunks > 0) {
        const size_t fbytes = (size_t)ns * m->g.field * sizeof(float);
        if (m->ut[0].ensure(fbytes) != FWI_OK || m->ut[1].ensure(fbytes) != FWI_OK) {
            cudaGetLastError();
            j.tb_chunks = 0;   // no room for the spare states: single steps
        }
    }
    return FWI_OK;
}

// The point work after forward step n has written u^{n+1} into `next`: the off-grid
// source taps, then the receiver samples (when traces are recorded).
int after_forward_step(fwi_model *m, const StepParams &p, float *next, int ns, int nr, int n,
                       float *traces, cudaStream_t s)
{
    const Geom &g = m->g;
    if (m->og_src)
        FWI_LAUNCH(m, launch_inject_pts(g, next, m->src_pts.as<PointTaps>(), ns, 1,
                                        m->W.as<float>(), sig_z(m), sig_y(m), sig_x(m),
                                        p.wavelet, m->nt, n, p.dt2, 0.0f, 0, s, p.n_dev));
    if (!traces) return FWI_OK;
    // the 3-D step sampled the receivers itself
    if (use_step3d(m) && m->rec_fuse_z >= 0 && !m->og_src && p.rec_tr == traces) return FWI_OK;
    if (m->og_rec)
        FWI_LAUNCH(m, launch_sample_pts(g, next, m->rec_pts.as<PointTaps>(), ns, nr, m->nt, n,
                                        traces, s, p.n_dev));
    else
        FWI_LAUNCH(m, launch_sample(g, next, m->rec_off.as<int64_t>(), ns, nr, m->nt, n, traces,
                                    s, p.n_dev));
    return FWI_OK;
}

// On completion u[cur] holds u^nt and u[1-cur] holds u^{nt-1}.
// Captures `units` forward steps (with their point work) from the current buffer parity
// into a graph that reads the step index from m->step_ctr and advances it.  On any
// failure the job falls back to issuing steps one by one.
int fwd_capture(FwdJob &j, int units)
{
    fwi_model *m = j.m;
    if (j.gexec) {
        cudaGraphExecDestroy(j.gexec);
        j.gexec = nullptr;
    }
    FWI_TRY(m->step_ctr.ensure(sizeof(int)));
    if (use_step3d(m)) ensure_resident(m);
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(j.s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        j.g_failed = true;
        return FWI_OK;
    }
    const int64_t l0 = m->launches;
    int rc = FWI_OK;
    StepParams p = j.p;
    p.n_dev = m->step_ctr.as<int>();
    float *uc = j.uc, *up = j.up;
    for (int i = 0; i < units && rc == FWI_OK; ++i) {
        p.cur = uc;
        p.prev = up;
        p.n = i;
        p.rec_tr = j.tr;
        ++m->launches;
        rc = raw_step(m, p, j.ns, false, j.s);
        if (rc == FWI_OK) rc = after_forward_step(m, p, p.prev, j.ns, j.nr, i, j.tr, j.s);
        std::swap(uc, up);
    }
    if (rc == FWI_OK) {
        ++m->launches;
        if (launch_tick(m->step_ctr.as<int>(), units, j.s) != cudaSuccess) rc = FWI_ERR_CUDA;
    }
    const cudaError_t ec = cudaStreamEndCapture(j.s, &graph);
    const int64_t nk = m->launches - l0;
    m->launches = l0;   // counted when the graph runs
    if (rc != FWI_OK || ec != cudaSuccess || !graph ||
        cudaGraphInstantiate(&j.gexec, graph, 0) != cudaSuccess) {
        cudaGetLastError();
        j.gexec = nullptr;
        j.g_failed = true;
    } else {
        j.g_units = units;
        j.g_uc = j.uc;
        j.g_kernels = nk;
    }
    if (graph) cudaGraphDestroy(graph);
    return FWI_OK;
}

// Temporal blocking on chip: up to 64 steps per cluster launch (k_step2d_cluster) from a
// one-entry table; the steps' arithmetic is the single step's.
int fwd_advance_onchip(FwdJob &j, int64_t units, bool *done)
{
    fwi_model *m = j.m;
    for (int64_t u = 0; u < units && j.n < m->nt;) {
        const int k = (int)std::min<int64_t>({units - u, (int64_t)(m->nt - j.n), 64});
        if (!m->cl_up) FWI_CU(cudaEventCreateWithFlags(&m->cl_up, cudaEventDisableTiming));
        FWI_CU(cudaEventSynchronize(m->cl_up));   // the staging is free again
        Batch2d *h = m->cl_host;
        h->count = 1;
        h->total_work = h->total_rec = 0;
        Batch2dEntry &e = h->e[0];
        e = Batch2dEntry{};
        e.p = j.p;
        e.p.n_dev = nullptr;
        e.u0 = j.uc;
        e.u1 = j.up;
        e.n0 = j.n;
        e.traces = j.tr;
        e.nrec = j.nr;
        e.rec_off = m->rec_off.as<int64_t>();
        e.rec_z = m->cl_rec_z;
        e.rec_x0 = m->cl_rec_x0;
        const int C = j.cl_size;
        const int smem = (int)((2LL * ((m->g.nz + C - 1) / C) * m->g.px * 4 + 1023) / 1024 * 1024);
        FWI_CU(cudaMemcpyAsync(m->cl_tab.p, h, offsetof(Batch2d, e) + sizeof(Batch2dEntry),
                               cudaMemcpyHostToDevice, j.s));
        FWI_CU(cudaEventRecord(m->cl_up, j.s));
        ++m->launches;
        FWI_CU(launch_step2d_cluster(m->cl_tab.as<Batch2d>(), m->M, k, C, 1, smem, j.s));
        if (k & 1) std::swap(j.uc, j.up);
        j.n += k;
        u += k;
    }
    *done = j.n >= m->nt;
    return FWI_OK;
}

int fwd_advance(FwdJob &j, int64_t units, bool *done)
{
    fwi_model *m = j.m;
    if (j.cl_size > 0) return fwd_advance_onchip(j, units, done);
    // a turn of an even number of steps (the serving loop's unit of work) replays one
    // captured graph: the buffer parity repeats after it and the step index comes from
    // the device counter
    if (units >= 2 && units <= 64 && units % 2 == 0 && m->nt - j.n >= units &&
        !m->opts.timing && !j.g_failed && j.tb_chunks == 0) {
        if (!j.gexec || j.g_units != units || j.g_uc != j.uc) FWI_TRY(fwd_capture(j, (int)units));
        if (j.gexec) {
            if (j.dev_n != j.n) {
                FWI_LAUNCH(m, launch_set_counter(m->step_ctr.as<int>(), j.n, j.s));
                j.dev_n = j.n;
            }
            FWI_CU(cudaGraphLaunch(j.gexec, j.s));
            m->launches += j.g_kernels;
            j.n += (int)units;
            j.dev_n += (int)units;
            *done = j.n >= m->nt;
            return FWI_OK;
        }
    }
    for (int64_t u = 0; u < units && j.n < m->nt;) {
        j.p.cur = j.uc;
        j.p.prev = j.up;
        j.p.n = j.n;
        if (j.tb_chunks > 0 && u + 2 <= units && j.n + 2 <= m->nt) {
            // two steps in one pass into the spare pair, which becomes the state
            float *o1 = (j.uc == m->u[0].as<float>() || j.uc == m->u[1].as<float>())
                            ? m->ut[0].as<float>() : m->u[0].as<float>();
            float *o2 = (o1 == m->ut[0].as<float>()) ? m->ut[1].as<float>() : m->u[1].as<float>();
            ++m->launches;
            FWI_CU(launch_step2d_tb2(j.p, j.ns, o1, o2, j.tb_chunks, j.s));
            FWI_TRY(after_forward_step(m, j.p, o1, j.ns, j.nr, j.n, j.tr, j.s));
            StepParams p1 = j.p;
            p1.n = j.n + 1;
            FWI_TRY(after_forward_step(m, p1, o2, j.ns, j.nr, j.n + 1, j.tr, j.s));
            j.up = o1;
            j.uc = o2;
            j.n += 2;
            u += 2;
            continue;
        }
        j.p.rec_tr = j.tr;
        FWI_TRY(step_launch(m, j.p, j.ns, false, 0, j.s));
        FWI_TRY(after_forward_step(m, j.p, j.p.prev, j.ns, j.nr, j.n, j.tr, j.s));
        std::swap(j.uc, j.up);
        ++j.n;
        ++u;
    }
    *done = j.n >= m->nt;
    return FWI_OK;
}

struct GradJob {
    fwi_model *m = nullptr;
    cudaStream_t s = nullptr;
    int ns = 0, nr = 0, nt = 0;
    int64_t nfield = 0;
    size_t fb = 0, half_slot = 0;   // bytes of one field's codes for all shots
    const void *dobs = nullptr;
    StepParams pf{}, pa{};
    float *tr = nullptr, *res = nullptr;
    int cur = 0, mcur = 0;
    int64_t step = 0, recorded = 0;
    std::vector<int64_t> slot_step;
    bool first_adj = true;
    int64_t nadj = 0, nfwd = 0, nstore = 0, nrestore = 0;
    const char *codes = nullptr;
    bool fused_max = false;
    size_t ia = 0;    // next schedule action
    int kdone = 0;    // forward steps already issued of the current ADVANCE action
    int aux_slot = -1;   // checkpoint the next reverse step reads u^m from in place
    int st_slot = -1, st_comps = 0;   // store the next forward step writes
    // CUDA graphs of kGradGraphSteps plain forward steps (no checkpoint store or max-abs
    // among them), keyed by the buffer parity at their start and whether they record
    // traces, replayed with the device step counter m->step_ctr (dev_n: its value as the
    // host last set it).  Used for turns of the serving loop.
    cudaGraphExec_t gx[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    int64_t gk[2][2] = {{0, 0}, {0, 0}};
    bool g_failed = false;
    int64_t dev_n = -1;
    GradJob() = default;
    GradJob(const GradJob &) = delete;
    GradJob &operator=(const GradJob &) = delete;
    ~GradJob()
    {
        for (auto &row : gx)
            for (auto &e : row)
                if (e) cudaGraphExecDestroy(e);
    }
};

constexpr int kGradGraphSteps = 8;

// Captures kGradGraphSteps forward steps from buffer parity `par`, recording traces when
// `rec`, into j.gx[par][rec]; a failed capture turns graphs off for the job.
int grad_capture(GradJob &j, int par, bool rec)
{
    fwi_model *m = j.m;
    FWI_TRY(m->step_ctr.ensure(sizeof(int)));
    if (use_step3d(m)) ensure_resident(m);
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(j.s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        j.g_failed = true;
        return FWI_OK;
    }
    const int64_t l0 = m->launches;
    int rc = FWI_OK;
    StepParams p = j.pf;
    p.n_dev = m->step_ctr.as<int>();
    p.maxbits = nullptr;
    p.st_code = nullptr;
    int cur = par;
    for (int i = 0; i < kGradGraphSteps && rc == FWI_OK; ++i) {
        p.cur = m->u[cur].as<float>();
        p.prev = m->u[1 - cur].as<float>();
        p.n = i;
        p.rec_tr = rec ? j.tr : nullptr;
        ++m->launches;
        rc = raw_step(m, p, j.ns, false, j.s);
        if (rc == FWI_OK)
            rc = after_forward_step(m, p, p.prev, j.ns, j.nr, i, rec ? j.tr : nullptr, j.s);
        cur = 1 - cur;
    }
    if (rc == FWI_OK) {
        ++m->launches;
        if (launch_tick(m->step_ctr.as<int>(), kGradGraphSteps, j.s) != cudaSuccess)
            rc = FWI_ERR_CUDA;
    }
    const cudaError_t ec = cudaStreamEndCapture(j.s, &graph);
    const int64_t nk = m->launches - l0;
    m->launches = l0;
    cudaGraphExec_t &gx = j.gx[par][rec ? 1 : 0];
    if (rc != FWI_OK || ec != cudaSuccess || !graph ||
        cudaGraphInstantiate(&gx, graph, 0) != cudaSuccess) {
        cudaGetLastError();
        gx = nullptr;
        j.g_failed = true;
    } else {
        j.gk[par][rec ? 1 : 0] = nk;
    }
    if (graph) cudaGraphDestroy(graph);
    return FWI_OK;
}

// Checkpoint slots for the budget, the schedule and its per-action component counts,
// staging of the inputs, and the initial state.

// The binomial schedule for nt steps and `slots` checkpoints, and the components each of
// its checkpoint actions moves (cached on the model per slot count).  A restore followed
// by a reverse step needs u^m alone (the reverse step reads only u^m, straight from the
// checkpoint; the following action is always another restore), and a checkpoint whose
// every restore is of that kind is stored as u^n alone.
// Code elements per shot in checkpoint slot k: two fields for a pair slot, else one.
int64_t slot_cstride(const fwi_model *m, int k) { return (m->slot_pair[k] ? 2 : 1) * m->g.field; }

template <class Plan>
void plan_schedule(Plan *m, int nt, int slots)
{
    if (slots == m->sched_nslots && m->sched_nt == nt) return;
    m->sched = revolve_actions(nt, (int32_t)slots, &m->sched_fwd);
    m->sched_nslots = slots;
    m->sched_nt = nt;
    const size_t na = m->sched.size() / 2;
    m->sched_comps.assign(na, 2);
    for (size_t i = 0; i < na; ++i) {
        const int kind = m->sched[2 * i], arg = m->sched[2 * i + 1];
        if (kind == 3 && arg >= 0 && i + 1 < na && m->sched[2 * (i + 1)] == 4)
            m->sched_comps[i] = 1;
    }
    // backwards: a store needs the pair if a pair restore of its slot follows it before
    // the slot's next store
    std::vector<char> need2(slots > 0 ? slots : 1, 0);
    m->slot_pair.assign(slots > 0 ? slots : 0, 0);
    for (size_t i = na; i-- > 0;) {
        const int kind = m->sched[2 * i], arg = m->sched[2 * i + 1];
        if (kind == 3 && arg >= 0 && m->sched_comps[i] == 2) need2[arg] = 1;
        if (kind == 2) {
            m->sched_comps[i] = need2[arg] ? 2 : 1;
            if (need2[arg]) m->slot_pair[arg] = 1;
            need2[arg] = 0;
        }
    }
    m->slot_off.assign(slots > 0 ? slots : 0, 0);
    int64_t off = 0;
    m->sched_npair = 0;
    for (int k = 0; k < slots; ++k) {
        m->slot_off[k] = off;
        off += m->slot_pair[k] ? 2 : 1;
        m->sched_npair += m->slot_pair[k] ? 1 : 0;
    }
}

// The largest slot count whose layout (slots that hold pairs count twice) fits `halves`
// units, never more than nt, by bisection (s slots fit, s + 1 do not); leaves that plan
// in *m.
template <class Plan>
int64_t fit_slots(Plan *m, int nt, int64_t halves)
{
    int64_t hi = halves < nt ? halves : nt;
    if (hi <= 0) {
        plan_schedule(m, nt, 0);
        return 0;
    }
    plan_schedule(m, nt, (int)hi);
    if (hi + m->sched_npair <= halves) return hi;
    int64_t lo = 0;   // no slots: no pairs, always fits
    while (hi - lo > 1) {
        const int64_t mid = lo + (hi - lo) / 2;
        plan_schedule(m, nt, (int)mid);
        if (mid + m->sched_npair <= halves) lo = mid;
        else hi = mid;
    }
    plan_schedule(m, nt, (int)lo);
    return lo;
}

int grad_setup(GradJob &j, fwi_model *m, const fwi_acq *acq, const float *wavelets,
               const float *d_obs, cudaStream_t s)
{
    j.m = m;
    j.s = s;
    const int ns = acq->nshots, nr = acq->nrec, nt = m->nt;
    j.ns = ns;
    j.nr = nr;
    j.nt = nt;
    FWI_TRY(ensure_workspace(m, acq, true, s));
    const Geom &g = m->g;
    j.nfield = (int64_t)ns * g.field;
    j.fb = (size_t)g.field * sizeof(float);

    // checkpoint slots: as many as the budget holds, never more than nt.  A checkpoint is
    // a pair (u^n and u^n - u^{n-1}) or u^n alone (every restore of it feeds a reverse
    // step), and the schedule fixes which: a slot takes two fields of codes per shot only
    // if it ever holds a pair, one otherwise.  The slot count is the largest whose layout
    // fits the budget; when u^n of every step fits, the schedule stores every state once
    // and never recomputes.
    const int esz = m->opts.snap_dtype == FWI_SNAP_FP32 ? 4 : 2;
    const size_t half_slot = (size_t)ns * g.field * esz;
    j.half_slot = half_slot;
    int64_t budget = m->opts.snap_budget_bytes;
    if (budget <= 0) {
        size_t fr = 0, tot = 0;
        FWI_CU(cudaMemGetInfo(&fr, &tot));
        budget = (int64_t)(fr / 4);
    }
    const void *pool0 = m->snaps.p;
    const size_t pool0_bytes = m->snaps.bytes;
    int64_t halves = budget / (int64_t)half_slot;
    int64_t slots = 0;
    for (;;) {
        slots = fit_slots(m, nt, halves);
        const size_t need = (size_t)(slots + m->sched_npair) * half_slot;
        // shrink on failure rather than fail: fewer slots only cost recomputation
        if (slots == 0 || need <= m->snaps.bytes || m->snaps.ensure(need) == FWI_OK) break;
        halves = (slots + m->sched_npair) * 7 / 8;
    }
    // zero the codes of the padding columns, which the stores of the step kernels skip,
    // whenever the pool is new or its layout changes (decoded padding must stay zero)
    const int64_t layout = ((int64_t)ns * g.field * 8191 + slots) * 8191 + m->sched_npair;
    const bool fresh = m->snaps.p != pool0 || m->snaps.bytes != pool0_bytes;
    if (m->snaps.p && (fresh || m->snaps_layout != layout)) {
        FWI_CU(cudaMemsetAsync(m->snaps.p, 0, m->snaps.bytes, s));
        m->snaps_layout = layout;
    }
    FWI_TRY(m->scales.ensure((size_t)(slots > 0 ? slots : 1) * 2 * ns * sizeof(float)));
    m->nslots = (int)slots;
    m->slot_bytes = slots > 0 ? (size_t)(slots + m->sched_npair) * half_slot / slots : 0;

    const void *wav;
    FWI_TRY(stage_input(m, 0, wavelets, (size_t)ns * nt * sizeof(float), s, &wav));
    FWI_TRY(stage_input(m, 1, d_obs, (size_t)ns * nt * nr * sizeof(float), s, &j.dobs));

    // adjoint receiver injection factor 2 W / a+ (the adjoint source is 2 r for Eq. 1)
    FWI_LAUNCH(m, launch_rec_scale(g, m->W.as<float>(), sig_z(m), sig_y(m), sig_x(m),
                                   m->rec_off.as<int64_t>(), ns * nr, 2.0f, 0,
                                   m->inj.as<float>(), s));
    FWI_CU(cudaMemsetAsync(m->u[0].p, 0, ns * j.fb, s));
    FWI_CU(cudaMemsetAsync(m->u[1].p, 0, ns * j.fb, s));
    FWI_CU(cudaMemsetAsync(m->g32.p, 0, ns * j.fb, s));
    FWI_CU(cudaMemsetAsync(m->g64.p, 0, ns * 2 * j.fb, s));

    j.pf = base_params(m);
    j.pf.src_off = m->og_src ? nullptr : m->src_off.as<int64_t>();
    j.pf.wavelet = (const float *)wav;
    j.pa = base_params(m);   // reverse sweep: receivers injected after each step; the
                             // wavelet enters only the imaging term at the source point
    j.pa.wavelet = (const float *)wav;
    j.tr = m->traces.as<float>();
    j.res = j.tr;            // residuals replace the traces in place
    j.slot_step.assign(slots > 0 ? slots : 1, -1);
    j.codes = m->snaps.as<char>();
    // the step kernels compute the checkpoint max-abs when asked, unless off-grid source
    // taps are added after the step (then a separate max-abs pass sees the final state)
    j.fused_max = !m->og_src;
    return FWI_OK;
}

int grad_advance(GradJob &j, int64_t units, bool *done)
{
    fwi_model *m = j.m;
    const Geom &g = m->g;
    const cudaStream_t s = j.s;
    const int ns = j.ns, nr = j.nr, nt = j.nt;
    const size_t nact = m->sched.size() / 2;
    int64_t used = 0;
    while (j.ia < nact && used < units) {
        const size_t ia = j.ia;
        const int kind = m->sched[2 * ia], arg = m->sched[2 * ia + 1];
        const int comps = m->sched_comps[ia];
        const bool next_store = ia + 1 < nact && m->sched[2 * (ia + 1)] == 2;
        if (kind == 1) {   // ADVANCE (may span several turns)
            while (j.kdone < arg && used < units) {
                // a serving turn replays a captured run of plain steps when the next
                // kGradGraphSteps steps hold no checkpoint store, no max-abs step and no
                // start or end of trace recording
                const int G = kGradGraphSteps;
                const int last_plain = arg - ((j.fused_max && next_store) ? 1 : 0);
                if (units <= 64 && !m->opts.timing && !j.g_failed && j.st_slot < 0 &&
                    j.kdone + G <= last_plain && units - used >= G &&
                    (j.step >= j.recorded) == (j.step + G - 1 >= j.recorded)) {
                    const int rec = j.step >= j.recorded ? 1 : 0;
                    if (!j.gx[j.cur][rec]) FWI_TRY(grad_capture(j, j.cur, rec != 0));
                    if (j.gx[j.cur][rec]) {
                        if (j.dev_n != j.step) {
                            FWI_LAUNCH(m, launch_set_counter(m->step_ctr.as<int>(), (int)j.step, s));
                            j.dev_n = j.step;
                        }
                        FWI_CU(cudaGraphLaunch(j.gx[j.cur][rec], s));
                        m->launches += j.gk[j.cur][rec];
                        j.step += G;
                        j.dev_n += G;
                        if (rec) j.recorded = j.step;
                        j.nfwd += G;
                        j.kdone += G;
                        used += G;
                        continue;
                    }
                }
                j.pf.cur = m->u[j.cur].as<float>();
                j.pf.prev = m->u[1 - j.cur].as<float>();
                j.pf.n = (int)j.step;
                j.pf.maxbits = nullptr;
                j.pf.st_code = nullptr;
                if (j.st_slot >= 0) {   // the deferred checkpoint of this step's input pair
                    j.pf.st_code = (void *)(j.codes + m->slot_off[j.st_slot] * j.half_slot);
                    j.pf.st_scale = m->scales.as<float>() + (size_t)j.st_slot * 2 * ns;
                    j.pf.st_dtype = m->opts.snap_dtype;
                    j.pf.st_comps = j.st_comps;
                    j.pf.st_cstride = slot_cstride(m, j.st_slot);
                    j.st_slot = -1;
                }
                if (j.fused_max && next_store && j.kdone == arg - 1) {
                    FWI_CU(cudaMemsetAsync(m->maxbits.p, 0, 2 * ns * sizeof(unsigned), s));
                    j.pf.maxbits = m->maxbits.as<unsigned>();
                }
                const bool rec_now = j.step >= j.recorded;
                j.pf.rec_tr = rec_now ? j.tr : nullptr;
                FWI_TRY(step_launch(m, j.pf, ns, false, j.pf.st_code ? 2 : 0, s));
                FWI_TRY(after_forward_step(m, j.pf, j.pf.prev, ns, nr, (int)j.step,
                                           rec_now ? j.tr : nullptr, s));
                if (rec_now) j.recorded = j.step + 1;
                j.cur = 1 - j.cur;
                ++j.step;
                ++j.nfwd;
                ++j.kdone;
                ++used;
            }
            if (j.kdone < arg) break;
            j.kdone = 0;
        } else if (kind == 2) {   // STORE the pair (u^step, u^{step-1}), or u^step alone
            const bool have_max = j.fused_max && ia > 0 && m->sched[2 * (ia - 1)] == 1;
            const bool next_adv = ia + 1 < nact && m->sched[2 * (ia + 1)] == 1;
            if (have_max && next_adv) {
                // the next forward step reads exactly this pair: it writes the checkpoint
                // from its epilogue with the scales derived here
                FWI_LAUNCH(m, launch_snap_scales(m->maxbits.as<unsigned>(), ns,
                                                 m->opts.snap_dtype,
                                                 m->scales.as<float>() + (size_t)arg * 2 * ns,
                                                 m->d_flag, s));
                j.st_slot = arg;
                j.st_comps = comps;
                j.slot_step[arg] = j.step;
                ++j.nstore;
                ++j.ia;
                continue;
            }
            if (!have_max) {
                FWI_CU(cudaMemsetAsync(m->maxbits.p, 0, 2 * ns * sizeof(unsigned), s));
                FWI_LAUNCH(m, launch_maxabs(m->u[j.cur].as<float>(), m->u[1 - j.cur].as<float>(),
                                            g.field, g.field, ns, m->maxbits.as<unsigned>(), s));
            }
            FWI_LAUNCH(m, launch_encode(m->u[j.cur].as<float>(), m->u[1 - j.cur].as<float>(),
                                        g.field, g.field, ns, m->opts.snap_dtype,
                                        m->maxbits.as<unsigned>(),
                                        (void *)(j.codes + m->slot_off[arg] * j.half_slot), slot_cstride(m, arg),
                                        m->scales.as<float>() + (size_t)arg * 2 * ns, m->d_flag,
                                        comps, s));
            j.slot_step[arg] = j.step;
            ++j.nstore;
        } else if (kind == 3) {   // RESTORE
            if (arg < 0) {
                FWI_CU(cudaMemsetAsync(m->u[0].p, 0, ns * j.fb, s));
                FWI_CU(cudaMemsetAsync(m->u[1].p, 0, ns * j.fb, s));
                j.cur = 0;
                j.step = 0;
            } else if (comps == 1) {
                // only the next reverse step needs this state, and it reads u^m from the
                // checkpoint in place: nothing to decode
                j.aux_slot = arg;
                j.step = j.slot_step[arg];
            } else {
                FWI_LAUNCH(m, launch_decode(j.codes + m->slot_off[arg] * j.half_slot, slot_cstride(m, arg),
                                            m->scales.as<float>() + (size_t)arg * 2 * ns, g.field,
                                            g.field, ns, m->opts.snap_dtype,
                                            m->u[j.cur].as<float>(),
                                            m->u[1 - j.cur].as<float>(), comps, s));
                j.step = j.slot_step[arg];
            }
            ++j.nrestore;
        } else if (kind == 4) {   // ADJOINT step m = arg, needs u^m = u[cur]
            const int mm = arg;
            if (j.step != mm)
                return fail(FWI_ERR_CUDA, "internal: checkpoint schedule out of step");
            if (j.first_adj) {
                // the receiver term of the imaging sum, from the traces before the misfit
                // turns them into residuals
                if (!m->og_rec)
                    FWI_LAUNCH(m, launch_rec_image(g, j.tr, (const float *)j.dobs,
                                                   m->rec_off.as<int64_t>(), ns, nr, nt,
                                                   m->g64.as<double>(), s));
                ++m->launches;   // the misfit is two launches
                FWI_LAUNCH(m, launch_misfit(j.tr, (const float *)j.dobs, j.res,
                                            (int64_t)ns * nt * nr, m->partials.as<double>(),
                                            misfit_blocks((int64_t)ns * nt * nr),
                                            m->phi.as<double>(), m->d_flag, s));
                FWI_CU(cudaMemsetAsync(m->mu[0].p, 0, ns * j.fb, s));
                FWI_CU(cudaMemsetAsync(m->mu[1].p, 0, ns * j.fb, s));
                j.first_adj = false;
            }
            j.pa.cur = m->mu[j.mcur].as<float>();        // mu^{m+1}
            j.pa.prev = m->mu[1 - j.mcur].as<float>();   // mu^{m+2} -> mu^m
            const bool img = mm < nt;                    // mu^{nt+1} = 0: no imaging at nt
            if (j.aux_slot >= 0) {                        // u^m from its checkpoint
                j.pa.aux = j.codes + m->slot_off[j.aux_slot] * j.half_slot;
                j.pa.aux_fmt = m->opts.snap_dtype;
                j.pa.aux_stride = slot_cstride(m, j.aux_slot);
                j.pa.aux_scale = m->scales.as<float>() + (size_t)j.aux_slot * 2 * ns;
            } else {                                      // u^m in the forward buffer
                j.pa.aux = m->u[j.cur].as<float>();
                j.pa.aux_fmt = FWI_SNAP_FP32;
                j.pa.aux_stride = g.field;
                j.pa.aux_scale = nullptr;
            }
            j.aux_slot = -1;
            j.pa.gacc = m->g32.as<float>();
            j.pa.src_off = (img && !m->og_src) ? m->src_off.as<int64_t>() : nullptr;
            j.pa.n = mm;
            // node receivers on one plane: the reverse step with imaging injects the
            // residual itself
            const bool inj_fused = img && use_step3d(m) && m->rec_fuse_z >= 0 && !m->og_rec;
            j.pa.inj_q = inj_fused ? j.res : nullptr;
            j.pa.inj_scale = m->inj.as<float>();
            j.pa.inj_n = mm - 1;
            FWI_TRY(step_launch(m, j.pa, ns, img, 1, s));
            if (img && m->og_src)   // source term of the imaging sum at the source taps
                FWI_LAUNCH(m, launch_image_pts(g, m->g32.as<float>(), j.pa.cur, 0, g.field,
                                               nullptr, m->src_pts.as<PointTaps>(), ns, 1,
                                               m->W.as<float>(), j.pa.wavelet, nt, mm,
                                               j.pa.dt2, 0, s));
            if (m->og_rec) {
                // receiver term of the imaging sum (u^m at the taps), then the injection
                FWI_LAUNCH(m, launch_image_pts(g, m->g32.as<float>(), j.pa.aux, j.pa.aux_fmt,
                                               j.pa.aux_stride, j.pa.aux_scale,
                                               m->rec_pts.as<PointTaps>(), ns * nr, nr,
                                               m->W.as<float>(), j.res, nt, mm - 1, j.pa.dt2,
                                               1, s));
                FWI_LAUNCH(m, launch_inject_pts(g, j.pa.prev, m->rec_pts.as<PointTaps>(),
                                                ns * nr, nr, m->W.as<float>(), sig_z(m),
                                                sig_y(m), sig_x(m), j.res, nt, mm - 1,
                                                j.pa.dt2, 2.0f, 1, s));
            } else if (!inj_fused) {
                FWI_LAUNCH(m, launch_inject(g, j.pa.prev, m->rec_off.as<int64_t>(),
                                            m->inj.as<float>(), j.res, ns, nr, nt, mm - 1, s));
            }
            if (mm == 1) {   // mu^1 is complete: the m = 0 source term of the imaging sum
                if (m->og_src)
                    FWI_LAUNCH(m, launch_image_pts(g, m->g32.as<float>(), j.pa.prev, 0, g.field,
                                                   nullptr, m->src_pts.as<PointTaps>(), ns, 1,
                                                   m->W.as<float>(), j.pa.wavelet, nt, 0,
                                                   j.pa.dt2, 0, s));
                else
                    FWI_LAUNCH(m, launch_src_image(g, j.pa.prev, m->src_off.as<int64_t>(),
                                                   m->W.as<float>(), j.pa.wavelet, j.pa.dt2, ns,
                                                   nt, m->g64.as<double>(), s));
            }
            j.mcur = 1 - j.mcur;
            ++j.nadj;
            ++used;
            if (j.nadj % m->opts.fold_every == 0)
                FWI_LAUNCH(m, launch_fold(m->g32.as<float>(), m->g64.as<double>(), j.nfield, s));
        }
        ++j.ia;
    }
    *done = j.ia >= nact;
    return FWI_OK;
}

// FP64 fold of the last partial gradient and the finish into the outputs (device targets
// of the caller or staging buffers; host copies are issued here).
int grad_finish(GradJob &j, double *misfit, float *grad, double *grad64, bool *sync_needed)
{
    fwi_model *m = j.m;
    const cudaStream_t s = j.s;
    FWI_LAUNCH(m, launch_fold(m->g32.as<float>(), m->g64.as<double>(), j.nfield, s));
    const int64_t nphys = m->np[0] * m->np[1] * m->np[2];
    void *g32dev = nullptr, *g64dev = nullptr;
    bool g32host = false, g64host = false;
    if (grad) FWI_TRY(output_target(m, 0, grad, nphys * sizeof(float), &g32dev, &g32host));
    if (grad64) FWI_TRY(output_target(m, 1, grad64, nphys * sizeof(double), &g64dev, &g64host));
    FWI_LAUNCH(m, launch_finish(m->g, m->nb, m->np, j.ns, m->g64.as<double>(), m->v.as<float>(),
                                (float *)g32dev, (double *)g64dev, s));
    FWI_TRY(finish_output(grad, g32dev, nphys * sizeof(float), g32host, s));
    FWI_TRY(finish_output(grad64, g64dev, nphys * sizeof(double), g64host, s));
    bool sync = g32host || g64host;
    if (misfit) {
        const bool mh = !is_device_ptr(misfit);
        FWI_CU(cudaMemcpyAsync(misfit, m->phi.p, sizeof(double),
                               mh ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
        sync = sync || mh;
    }
    m->st_fwd = j.nfwd;
    m->st_adj = j.nadj;
    m->st_store = j.nstore;
    m->st_restore = j.nrestore;
    *sync_needed = sync;
    return FWI_OK;
}

// ---- opaque jobs for the serving loop (jobs.h)

struct Job {
    int kind = 0;   // 0 forward, 1 gradient
    FwdJob f;
    GradJob gj;
    int nrec = 0;
    int row_z = -2, row_x0 = 0;   // receivers as one row (row_z >= 0), -1: not, -2: unknown
};

Job *job_forward(fwi_model *m, const fwi_acq *acq, const float *wavelets, cudaStream_t s,
                 int *rc)
{
    *rc = validate_acq(m, acq);
    if (*rc != FWI_OK) return nullptr;
    *rc = ensure_workspace(m, acq, false, s);
    if (*rc != FWI_OK) return nullptr;
    const void *wav;
    *rc = stage_input(m, 0, wavelets, (size_t)acq->nshots * m->nt * sizeof(float), s, &wav);
    if (*rc != FWI_OK) return nullptr;
    Job *j = new Job();
    j->kind = 0;
    j->nrec = acq->nrec;
    *rc = fwd_setup(j->f, m, acq->nshots, acq->nrec, (const float *)wav, m->traces.as<float>(), s);
    if (*rc != FWI_OK) {
        delete j;
        return nullptr;
    }
    return j;
}

Job *job_gradient(fwi_model *m, const fwi_acq *acq, const float *wavelets, const float *d_obs,
                  cudaStream_t s, int *rc)
{
    *rc = validate_acq(m, acq);
    if (*rc != FWI_OK) return nullptr;
    Job *j = new Job();
    j->kind = 1;
    j->nrec = acq->nrec;
    *rc = grad_setup(j->gj, m, acq, wavelets, d_obs, s);
    if (*rc != FWI_OK) {
        delete j;
        return nullptr;
    }
    return j;
}

int job_advance(Job *j, int64_t units, bool *done)
{
    return j->kind == 0 ? fwd_advance(j->f, units, done) : grad_advance(j->gj, units, done);
}

// The serving loop's shared 2-D forward launch.  A forward job of one 2-D shot with a
// node source and node receivers (no temporal blocking, no kernel timing) may have its
// time steps issued by k_step2d_multi instead of job_advance: job_batch_entry fills a
// table entry with its state, job_batch_moved records that `steps` steps ran.
bool job_batchable(const Job *j)
{
    if (j->kind != 0) return false;
    const fwi_model *m = j->f.m;
    return m->ndim == 2 && j->f.ns == 1 && !m->og_src && !m->og_rec && j->f.tb_chunks == 0 &&
           !m->opts.timing && j->f.tr != nullptr;
}

int job_batch_entry(Job *j, Batch2dEntry *e, int zchunk)
{
    if (!job_batchable(j)) return fail(FWI_ERR_ARG, "job not eligible for the shared launch");
    const FwdJob &f = j->f;
    const fwi_model *m = f.m;
    if (j->row_z == -2) {
        // receivers that are consecutive nodes of one row are sampled by the step itself
        j->row_z = -1;
        const int nr = f.nr;
        if (nr > 0 && (int64_t)m->geo_rec.size() >= 3 * (int64_t)nr) {
            const int64_t o0 = node_offset(m, m->geo_rec.data());
            const int z = (int)(o0 / m->g.plane), x0 = (int)(o0 - (int64_t)z * m->g.plane);
            bool row = x0 + nr <= m->g.nx;
            for (int r = 1; row && r < nr; ++r) row = node_offset(m, m->geo_rec.data() + 3 * r) == o0 + r;
            if (row) {
                j->row_z = z;
                j->row_x0 = x0;
            }
        }
    }
    e->p = f.p;
    e->p.zchunk = zchunk;
    e->p.nzchunks = (m->g.nz + zchunk - 1) / zchunk;
    e->p.n_dev = nullptr;
    e->u0 = f.uc;
    e->u1 = f.up;
    e->n0 = f.n;
    e->xtiles = (m->g.nx + 255) / 256;
    e->rec_off = m->rec_off.as<int64_t>();
    e->traces = f.tr;
    e->nrec = f.nr;
    e->rec_z = j->row_z;
    e->rec_x0 = j->row_x0;
    e->nsamp = j->row_z >= 0 ? 0 : f.nr;
    return FWI_OK;
}

int job_batch_moved(Job *j, int steps, bool *done)
{
    FwdJob &f = j->f;
    const int left = f.m->nt - f.n;
    const int moved = steps < left ? steps : left;
    if (moved & 1) std::swap(f.uc, f.up);
    f.n += moved;
    f.m->launches += 2 * (int64_t)moved;
    *done = f.n >= f.m->nt;
    return FWI_OK;
}

// Issues the result copies into host buffers (traces [ns][nt][nrec] of a forward job, or
// misfit and gradient of a gradient job) on the job's stream; the caller synchronises.
int job_finish(Job *j, double *misfit_host, float *out_host)
{
    if (j->kind == 0) {
        fwi_model *m = j->f.m;
        if (out_host)
            FWI_CU(cudaMemcpyAsync(out_host, m->traces.p,
                                   (size_t)j->f.ns * m->nt * j->nrec * sizeof(float),
                                   cudaMemcpyDeviceToHost, j->f.s));
        return FWI_OK;
    }
    bool sync = false;
    return grad_finish(j->gj, misfit_host, out_host, nullptr, &sync);
}

void job_free(Job *j) { delete j; }

}  // namespace fwi

// ====================================================================== C ABI

extern "C" {

const char *fwi_last_error(void) { return g_err.c_str(); }

int fwi_fd_coeffs(int32_t order, double *c)
{
    if (!c || order % 2 || order < 2 || order > 2 * kMaxM)
        return fail(FWI_ERR_ARG, "order must be even, 2..16");
    return host_coeffs(order / 2, c);
}

double fwi_cfl_number(int32_t ndim, int32_t order, const float spacing[3], float vmax, float dt)
{
    if ((ndim != 2 && ndim != 3) || order % 2 || order < 2 || order > 2 * kMaxM || !spacing)
        return -1.0;
    return host_cfl(ndim, order / 2, spacing, vmax, dt);
}

int fwi_revolve_schedule(int32_t nsteps, int32_t nslots, int32_t *actions,
                         int64_t max_actions, int64_t *n_actions, int64_t *n_forward)
{
    if (nsteps < 1 || nslots < 0) return fail(FWI_ERR_ARG, "nsteps >= 1 and nslots >= 0");
    int64_t fwd = 0;
    std::vector<int32_t> a = revolve_actions(nsteps, nslots, &fwd);
    const int64_t na = (int64_t)a.size() / 2;
    if (n_actions) *n_actions = na;
    if (n_forward) *n_forward = fwd;
    if (!actions) return FWI_OK;
    if (na > max_actions) return fail(FWI_ERR_ARG, "max_actions too small");
    std::memcpy(actions, a.data(), a.size() * sizeof(int32_t));
    return FWI_OK;
}

int fwi_checkpoint_plan(int32_t nsteps, int64_t half_slots, int32_t *slots,
                        int32_t *pair_slots, int64_t *n_forward)
{
    if (nsteps < 1 || half_slots < 0) return fail(FWI_ERR_ARG, "nsteps >= 1 and half_slots >= 0");
    struct {
        std::vector<int32_t> sched;
        std::vector<int> sched_comps;
        int64_t sched_fwd = 0;
        int sched_nslots = -1, sched_nt = -1, sched_npair = 0;
        std::vector<int64_t> slot_off;
        std::vector<char> slot_pair;
    } plan;
    const int64_t n = fit_slots(&plan, nsteps, half_slots);
    if (slots) *slots = (int32_t)n;
    if (pair_slots) *pair_slots = plan.sched_npair;
    if (n_forward) *n_forward = plan.sched_fwd;
    return FWI_OK;
}

int fwi_create_model(fwi_model **out, int32_t ndim, const int64_t shape[3],
                     const float spacing[3], const float *vp, float dt, int32_t nt,
                     const fwi_opts *opts, cudaStream_t stream)
{
    if (!out || !shape || !spacing || !vp) return fail(FWI_ERR_ARG, "null argument");
    *out = nullptr;
    if (ndim != 2 && ndim != 3) return fail(FWI_ERR_ARG, "ndim must be 2 or 3");
    if (shape[0] < 1 || shape[1] < 1 || shape[2] < 1 || (ndim == 2 && shape[1] != 1))
        return fail(FWI_ERR_ARG, "shape must be positive (ny = 1 in 2-D)");
    if (!(dt > 0.0f) || nt < 1) return fail(FWI_ERR_ARG, "dt > 0 and nt >= 1 required");
    for (int a = 0; a < 3; ++a)
        if ((a != 1 || ndim == 3) && !(spacing[a] > 0.0f))
            return fail(FWI_ERR_ARG, "spacing must be positive");
    fwi_opts o{};
    if (opts) o = *opts;
    if (o.order == 0) o.order = 8;
    if (o.order != 8 && o.order != 16) return fail(FWI_ERR_ARG, "order must be 8 or 16");
    if (o.nb == 0) o.nb = 20;
    if (o.nb < 0) o.nb = 0;
    if (o.snap_dtype < 0 || o.snap_dtype > 2) return fail(FWI_ERR_ARG, "bad snap_dtype");
    // the FP32 gradient accumulator is folded into FP64 every 256 reverse steps: measured on
    // the 96^3 salt twin (600 steps, FP32 checkpoints) the gradient's error against the
    // FP64 oracle is 2.8e-5 with a fold every 64, 256 or 1024 steps, or none
    if (o.fold_every <= 0) o.fold_every = 256;
    if (!(o.sponge_r0 > 0.0f)) o.sponge_r0 = 1e-3f;
    if (o.sponge_r0 >= 1.0f) return fail(FWI_ERR_ARG, "sponge_r0 must be in (0, 1)");

    fwi_model *m = new fwi_model();
    m->ndim = ndim;
    m->order = o.order;
    m->M = o.order / 2;
    m->nb = o.nb;
    m->nt = nt;
    m->dt = dt;
    m->opts = o;
    for (int a = 0; a < 3; ++a) {
        m->np[a] = shape[a];
        m->h[a] = (a == 1 && ndim == 2) ? 1.0f : spacing[a];
    }
    Geom &g = m->g;
    g.ndim = ndim;
    g.M = m->M;
    const int64_t nz = shape[0] + 2 * o.nb, ny = ndim == 3 ? shape[1] + 2 * o.nb : 1,
                  nx = shape[2] + 2 * o.nb;
    if (nz > (1 << 30) || ny > (1 << 30) || nx > (1 << 30) || nz * ny >= ((int64_t)1 << 31)) {
        delete m;
        return fail(FWI_ERR_ARG, "grid too large");
    }
    g.nz = (int)nz;
    g.ny = (int)ny;
    g.nx = (int)nx;
    g.px = (int)round_up(nx, 8);
    g.plane = (int64_t)g.ny * g.px;
    g.field = round_up((int64_t)g.nz * g.plane, 64);
    int rc = set_coefs(m);
    if (rc == FWI_OK) {
        cudaError_t e = cudaHostAlloc((void **)&m->h_flag, sizeof(unsigned), cudaHostAllocMapped);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&m->d_flag, m->h_flag, 0);
        if (e != cudaSuccess) {
            cudaGetLastError();
            rc = fail(FWI_ERR_CUDA, std::string("status word: ") + cudaGetErrorString(e));
        } else {
            *m->h_flag = 0;
        }
    }
    if (rc == FWI_OK) rc = set_velocity(m, vp, stream);
    if (rc != FWI_OK) {
        std::string msg = g_err;
        fwi_destroy(m);
        g_err = msg;
        return rc;
    }
    m->last_stream = stream;
    *out = m;
    return FWI_OK;
}

int fwi_update_velocity(fwi_model *m, const float *vp, cudaStream_t stream)
{
    if (!m || !vp) return fail(FWI_ERR_ARG, "null argument");
    m->last_stream = stream;
    return set_velocity(m, vp, stream);
}

int fwi_forward(fwi_model *m, const fwi_acq *acq, const float *wavelets, float *traces,
                float *final_state, cudaStream_t s)
{
    if (!m || !wavelets) return fail(FWI_ERR_ARG, "null argument");
    FWI_TRY(check_status(m));
    FWI_TRY(validate_acq(m, acq));
    m->last_stream = s;
    const int ns = acq->nshots, nr = acq->nrec;
    FWI_TRY(ensure_workspace(m, acq, false, s));
    const void *wav;
    FWI_TRY(stage_input(m, 0, wavelets, (size_t)ns * m->nt * sizeof(float), s, &wav));
    void *trdev = nullptr;
    bool trhost = false;
    const size_t trbytes = (size_t)ns * m->nt * nr * sizeof(float);
    if (traces) FWI_TRY(output_target(m, 0, traces, trbytes, &trdev, &trhost));
    FwdJob job;
    FWI_TRY(fwd_setup(job, m, ns, nr, (const float *)wav, (float *)trdev, s));
    bool done = false;
    FWI_TRY(fwd_advance(job, INT64_MAX, &done));
    FWI_LAUNCH(m, launch_nonfinite_check(job.uc, (int64_t)ns * m->g.field, m->d_flag, s));
    bool sync = trhost;
    if (final_state) {
        const bool fhost = !is_device_ptr(final_state);
        const int64_t pts = (int64_t)m->g.nz * m->g.ny * m->g.nx;
        for (int sh = 0; sh < ns; ++sh)
            for (int k = 0; k < 2; ++k) {
                const float *srcp = (k == 0 ? job.uc : job.up) + (int64_t)sh * m->g.field;
                float *dst = final_state + ((int64_t)sh * 2 + k) * pts;
                FWI_CU(cudaMemcpy2DAsync(dst, m->g.nx * sizeof(float), srcp, m->g.px * sizeof(float),
                                         m->g.nx * sizeof(float), (size_t)m->g.nz * m->g.ny,
                                         fhost ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
            }
        sync = sync || fhost;
    }
    FWI_TRY(finish_output(traces, trdev, trbytes, trhost, s));
    if (sync) {
        FWI_CU(cudaStreamSynchronize(s));
        FWI_TRY(check_status(m));
    }
    FWI_TRY(collect_timing(m));
    return FWI_OK;
}

int fwi_adjoint_gradient(fwi_model *m, const fwi_acq *acq, const float *wavelets,
                         const float *d_obs, double *misfit, float *grad, double *grad64,
                         cudaStream_t s)
{
    if (!m || !wavelets || !d_obs) return fail(FWI_ERR_ARG, "null argument");
    FWI_TRY(check_status(m));
    FWI_TRY(validate_acq(m, acq));
    m->last_stream = s;
    GradJob job;
    FWI_TRY(grad_setup(job, m, acq, wavelets, d_obs, s));
    bool done = false;
    FWI_TRY(grad_advance(job, INT64_MAX, &done));
    bool sync = false;
    FWI_TRY(grad_finish(job, misfit, grad, grad64, &sync));
    if (sync) {
        FWI_CU(cudaStreamSynchronize(s));
        FWI_TRY(check_status(m));
    }
    FWI_TRY(collect_timing(m));
    return FWI_OK;
}

int fwi_source_adjoint(fwi_model *m, const fwi_acq *acq, const float *y, float *x,
                       cudaStream_t s)
{
    if (!m || !y || !x) return fail(FWI_ERR_ARG, "null argument");
    FWI_TRY(check_status(m));
    FWI_TRY(validate_acq(m, acq));
    m->last_stream = s;
    const int ns = acq->nshots, nr = acq->nrec, nt = m->nt;
    FWI_TRY(ensure_workspace(m, acq, true, s));
    const Geom &g = m->g;
    const size_t fb = (size_t)g.field * sizeof(float);
    const void *ydev;
    FWI_TRY(stage_input(m, 0, y, (size_t)ns * nt * nr * sizeof(float), s, &ydev));
    void *xdev;
    bool xhost;
    FWI_TRY(output_target(m, 0, x, (size_t)ns * nt * sizeof(float), &xdev, &xhost));
    // injection W y / a+ at the receivers; read-out dt^2 mu / W at the source
    FWI_LAUNCH(m, launch_rec_scale(g, m->W.as<float>(), sig_z(m), sig_y(m), sig_x(m),
                            m->rec_off.as<int64_t>(), ns * nr, 1.0f, 0, m->inj.as<float>(), s));
    FWI_LAUNCH(m, launch_rec_scale(g, m->W.as<float>(), sig_z(m), sig_y(m), sig_x(m),
                            m->src_off.as<int64_t>(), ns, m->dt * m->dt, 1,
                            m->src_scale.as<float>(), s));
    FWI_CU(cudaMemsetAsync(m->mu[0].p, 0, ns * fb, s));
    FWI_CU(cudaMemsetAsync(m->mu[1].p, 0, ns * fb, s));
    StepParams pa = base_params(m);
    int mcur = 0;
    for (int mm = nt; mm >= 1; --mm) {
        pa.cur = m->mu[mcur].as<float>();
        pa.prev = m->mu[1 - mcur].as<float>();
        FWI_TRY(step_launch(m, pa, ns, false, 1, s));
        if (m->og_rec)
            FWI_LAUNCH(m, launch_inject_pts(g, pa.prev, m->rec_pts.as<PointTaps>(), ns * nr, nr,
                                            m->W.as<float>(), sig_z(m), sig_y(m), sig_x(m),
                                            (const float *)ydev, nt, mm - 1, pa.dt2, 1.0f, 1, s));
        else
            FWI_LAUNCH(m, launch_inject(g, pa.prev, m->rec_off.as<int64_t>(), m->inj.as<float>(),
                                        (const float *)ydev, ns, nr, nt, mm - 1, s));
        if (m->og_src)
            FWI_LAUNCH(m, launch_gather_src_pts(g, pa.prev, m->src_pts.as<PointTaps>(), ns,
                                                m->W.as<float>(), pa.dt2, nt, mm - 1,
                                                (float *)xdev, s));
        else
            FWI_LAUNCH(m, launch_gather_src(g, pa.prev, m->src_off.as<int64_t>(),
                                            m->src_scale.as<float>(), ns, nt, mm - 1,
                                            (float *)xdev, s));
        mcur = 1 - mcur;
    }
    FWI_TRY(finish_output(x, xdev, (size_t)ns * nt * sizeof(float), xhost, s));
    if (xhost) FWI_CU(cudaStreamSynchronize(s));
    FWI_TRY(collect_timing(m));
    return FWI_OK;
}

int fwi_misfit(const float *d_mod, const float *d_obs, int64_t n, double *misfit_dev,
               cudaStream_t s)
{
    if (!d_mod || !d_obs || !misfit_dev || n < 0) return fail(FWI_ERR_ARG, "bad argument");
    const int nb = misfit_blocks(n);
    double *part = nullptr;
    FWI_CU(cudaMallocAsync((void **)&part, nb * sizeof(double), s));
    cudaError_t e = launch_misfit(d_mod, d_obs, nullptr, n, part, nb, misfit_dev, nullptr, s);
    cudaError_t e2 = cudaFreeAsync(part, s);
    if (e != cudaSuccess) return fail(FWI_ERR_CUDA, std::string("misfit: ") + cudaGetErrorString(e));
    if (e2 != cudaSuccess) return fail(FWI_ERR_CUDA, std::string("misfit free: ") + cudaGetErrorString(e2));
    return FWI_OK;
}

int fwi_snapshot_encode(const float *a, const float *b, int64_t n, int32_t dtype, void *code,
                        float *scale, cudaStream_t s)
{
    if (!a || !b || !code || !scale || n < 0 || dtype < 0 || dtype > 2)
        return fail(FWI_ERR_ARG, "bad argument");
    unsigned *mb = nullptr;
    FWI_CU(cudaMallocAsync((void **)&mb, 2 * sizeof(unsigned), s));
    FWI_CU(cudaMemsetAsync(mb, 0, 2 * sizeof(unsigned), s));
    cudaError_t e = launch_maxabs(a, b, n, n, 1, mb, s);
    if (e == cudaSuccess) e = launch_encode(a, b, n, n, 1, dtype, mb, code, 2 * n, scale, nullptr, 2, s);
    cudaError_t e2 = cudaFreeAsync(mb, s);
    if (e != cudaSuccess || e2 != cudaSuccess)
        return fail(FWI_ERR_CUDA, std::string("encode: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    return FWI_OK;
}

int fwi_snapshot_decode(const void *code, const float *scale, int64_t n, int32_t dtype, float *a,
                        float *b, cudaStream_t s)
{
    if (!a || !b || !code || !scale || n < 0 || dtype < 0 || dtype > 2)
        return fail(FWI_ERR_ARG, "bad argument");
    FWI_CU(launch_decode(code, 2 * n, scale, n, n, 1, dtype, a, b, 2, s));
    return FWI_OK;
}

int fwi_model_info(const fwi_model *m, fwi_info *o)
{
    if (!m || !o) return fail(FWI_ERR_ARG, "null argument");
    std::memset(o, 0, sizeof(*o));
    o->ndim = m->ndim;
    o->order = m->order;
    o->nb = m->nb;
    o->nt = m->nt;
    for (int a = 0; a < 3; ++a) o->shape[a] = m->np[a];
    o->computed[0] = m->g.nz;
    o->computed[1] = m->g.ny;
    o->computed[2] = m->g.nx;
    o->pitch_x = m->g.px;
    o->points = (int64_t)m->g.nz * m->g.ny * m->g.nx;
    o->device_bytes = m->device_bytes();
    o->snap_slots = m->nslots;
    o->shots_capacity = m->cap_shots;
    o->last_forward_steps = m->st_fwd;
    o->last_adjoint_steps = m->st_adj;
    o->last_snap_stores = m->st_store;
    o->last_snap_restores = m->st_restore;
    for (int a = 0; a < 3; ++a) o->sponge_eta_max[a] = m->eta_max[a];
    o->cfl = m->cfl;
    o->kernel_launches = m->launches;
    o->fwd_step_launches = m->t_fwd_n;
    o->adj_step_launches = m->t_adj_n;
    o->fwd_step_ms = m->t_fwd_ms;
    o->adj_step_ms = m->t_adj_ms;
    o->store_step_launches = m->t_st_n;
    o->store_step_ms = m->t_st_ms;
    // modes in the order forward, reverse, forward + store
    const int mode_of[3] = {kModeStep, kModeAdj, kModeStepStore};
    for (int k = 0; k < 3; ++k) {
        const int q = m->resident_query[mode_of[k]];
        o->step_ctas[k] = q < 0 ? q : m->resident[mode_of[k]];
    }
    o->reserved2 = 0;
    return FWI_OK;
}

int fwi_selftest_wait(fwi_model *m, int32_t polls, cudaStream_t s)
{
    if (!m) return fail(FWI_ERR_ARG, "null argument");
    if (polls < 1 || polls > (1 << 22))
        return fail(FWI_ERR_ARG, "fwi_selftest_wait: polls must lie in [1, 2^22]");
    m->last_stream = s;
    FWI_LAUNCH(m, launch_wait_selftest(m->d_flag, polls, s));
    return FWI_OK;
}

int fwi_sync_status(fwi_model *m)
{
    if (!m) return fail(FWI_ERR_ARG, "null argument");
    FWI_CU(cudaStreamSynchronize(m->last_stream));
    return check_status(m);
}

void fwi_destroy(fwi_model *m)
{
    if (!m) return;
    if (m->last_stream) cudaStreamSynchronize(m->last_stream);
    m->v.release();
    m->W.release();
    m->sig.release();
    for (int i = 0; i < 2; ++i) {
        m->u[i].release();
        m->mu[i].release();
        m->stage_out[i].release();
    }
    for (int i = 0; i < 3; ++i) m->stage_in[i].release();
    m->g32.release();
    m->g64.release();
    m->traces.release();
    m->src_off.release();
    m->rec_off.release();
    m->inj.release();
    m->src_scale.release();
    m->maxbits.release();
    m->partials.release();
    m->phi.release();
    m->snaps.release();
    m->scales.release();
    if (m->h_flag) cudaFreeHost(m->h_flag);
    m->cl_tab.release();
    m->rec_map.release();
    if (m->cl_host) cudaFreeHost(m->cl_host);
    if (m->cl_up) cudaEventDestroy(m->cl_up);
    for (cudaEvent_t e : m->ev) cudaEventDestroy(e);
    delete m;
}

}  // extern "C"
