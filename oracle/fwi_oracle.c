/*
 * FP64 CPU oracle for acoustic full-waveform inversion: forward modelling, exact
 * discrete adjoint and the zero-lag imaging condition (velocity gradient).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls this
 * file; only the tests, the package's smoke check and the CPU baseline of the bench
 * do.  It shares no code, header, table or helper with the CUDA library: the
 * finite-difference coefficients, the sponge profile, the CFL number and every
 * update below are derived here again from their definitions.
 *
 * Every function is a plain loop over the grid in double precision, in the order the
 * method states it, with no blocking, fusion or reordering beyond that.  OpenMP only
 * splits the outermost grid loop.
 *
 * Sources of each definition ("HRI" = Huot et al., High-resolution imaging on TPUs):
 *   - misfit  phi = || d_mod - d_obs ||_2^2                      HRI Sec. 3, Eq. 1
 *   - wave equation  P_tt = v^2 lap(P) + s                       HRI Sec. 3, Eq. 2
 *   - leapfrog update P^{n+1} = -P^{n-1} + 2P^n + v^2 dt^2 lap P^n + dt^2 s^n
 *                                                                HRI Sec. 3, Eq. 3
 *   - central stencils of order >= 8 (8th and 16th used)         HRI Sec. 3 (Fig. 3), Sec. 4
 *   - the gradient of phi (named, not derived, in the paper)     HRI Sec. 1
 * Readings where the paper is silent (all stated again where they are used):
 *   - coefficients: Taylor (Fornberg) central second-derivative weights of radius M,
 *     order 2M;
 *   - absorbing boundary: a damped wave equation P_tt + eta P_t = v^2 lap P + s with a
 *     quadratic sponge of nb cells padded outside the physical grid on every face,
 *     centred in time, which reduces to Eq. 3 wherever eta = 0;
 *   - outside the padded (computed) grid the field is zero (Dirichlet);
 *   - source: dt^2 w[n] added at one node (Eq. 3's dt^2 s term), divided by the same
 *     a+ factor as the rest of the update;
 *   - receivers: sample n of a trace is the field after step n, u^{n+1};
 *   - off-grid sources and receivers (an extension; the paper places them on nodes):
 *     Kaiser-windowed sinc interpolation (Hicks 2002, Geophysics 67(1), 156-166),
 *     half-width 4 and b = 6.31, used for sampling and, transposed, for injection;
 *   - quiescent start u^{-1} = u^0 = 0;
 *   - gradient: exact derivative of the discrete phi with respect to the physical
 *     velocity grid, with the sponge strength held fixed; sponge cells take the
 *     velocity of the nearest physical cell (edge replication), so their
 *     contributions fold back onto that cell.
 *
 * Parity status: every function here is pinned by the CPU tests (coefficients by
 * exact rational moment conditions, the Laplacian by its convergence order and
 * modified-wavenumber symbol, time stepping by closed-box energy conservation and the
 * homogeneous Green's function, the adjoint by dot-product tests and the gradient by
 * central finite differences).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXM 8

/* ------------------------------------------------------------------ coefficients */

/* Central second-derivative weights of radius M (order 2M): the unique symmetric
 * stencil that is exact for polynomials up to degree 2M+1.  Closed form
 *   c_k = 2 (-1)^{k+1} (M!)^2 / (k^2 (M-k)! (M+k)!),  k = 1..M,
 *   c_0 = -2 sum_k c_k.
 * The factorials stay below 2^53 for M <= 8, so every factor is exact in double. */
int oracle_fd_coeffs(int M, double *c)
{
    if (M < 1 || M > OR_MAXM) return -1;
    double fM = 1.0;
    for (int i = 2; i <= M; ++i) fM *= i;
    double sum = 0.0;
    for (int k = 1; k <= M; ++k) {
        double fa = 1.0, fb = 1.0;
        for (int i = 2; i <= M - k; ++i) fa *= i;
        for (int i = 2; i <= M + k; ++i) fb *= i;
        double sgn = (k % 2 == 1) ? 1.0 : -1.0;
        c[k] = 2.0 * sgn * (fM / fa) * (fM / fb) / ((double)k * (double)k);
        sum += c[k];
    }
    c[0] = -2.0 * sum;
    return 0;
}

/* Stability number of the undamped leapfrog: the scheme is stable while
 *   v_max dt sqrt(sum_axes S_M / h_a^2) / 2 < 1,
 * where S_M = -(c_0 + 2 sum_k c_k cos(k pi)) is the largest eigenvalue magnitude of
 * the 1-D stencil (its symbol at the Nyquist wavenumber). */
double oracle_cfl_number(int ndim, int M, const double *h, double vmax, double dt)
{
    double c[OR_MAXM + 1];
    if (oracle_fd_coeffs(M, c) != 0) return -1.0;
    double S = -c[0];
    for (int k = 1; k <= M; ++k) S -= 2.0 * c[k] * ((k % 2 == 0) ? 1.0 : -1.0);
    double acc = S / (h[0] * h[0]) + S / (h[2] * h[2]);
    if (ndim == 3) acc += S / (h[1] * h[1]);
    return vmax * dt * sqrt(acc) / 2.0;
}

/* ------------------------------------------------------------------ grid */

typedef struct {
    int ndim, M, nb;
    int64_t np[3];  /* physical extents (nz, ny, nx); ny = 1 in 2-D */
    int64_t n[3];   /* computed (padded) extents */
    int64_t ncell;
    double h[3];
    double dt;
    double c[OR_MAXM + 1];
    double *W;      /* v_c^2 dt^2 on the computed grid */
    double *vc;     /* edge-replicated velocity */
    double *ap, *am;/* a+ = 1 + eta dt / 2, a- = 1 - eta dt / 2 */
} og_grid;

static int64_t og_clamp(int64_t i, int64_t lo, int64_t hi)
{
    return i < lo ? lo : (i > hi ? hi : i);
}

/* depth of index i into the sponge of an axis of physical extent np, padded by nb */
static double og_depth(int64_t i, int64_t np, int nb)
{
    if (i < nb) return (double)(nb - i);
    if (i >= nb + np) return (double)(i - (nb + np - 1));
    return 0.0;
}

static void og_free(og_grid *g)
{
    free(g->W); free(g->vc); free(g->ap); free(g->am);
    g->W = g->vc = g->ap = g->am = NULL;
}

/* Builds the computed grid: pads v by nb cells on every face of every present axis by
 * edge replication, W = v_c^2 dt^2, and the sponge
 *   eta = sum_axes eta_max,a (depth_a / nb)^2,
 *   eta_max,a = 3 vref ln(1/R0) / (2 nb h_a)
 * (vref <= 0 means the largest velocity of the model). */
static int og_build(og_grid *g, int ndim, const int64_t *shape, const double *h,
                    const double *v, double dt, int M, int nb, double r0, double vref)
{
    memset(g, 0, sizeof(*g));
    if (ndim != 2 && ndim != 3) return -1;
    if (oracle_fd_coeffs(M, g->c) != 0) return -1;
    g->ndim = ndim; g->M = M; g->nb = nb; g->dt = dt;
    for (int a = 0; a < 3; ++a) { g->np[a] = shape[a]; g->h[a] = h[a]; }
    if (ndim == 2) g->np[1] = 1;
    g->n[0] = g->np[0] + 2 * nb;
    g->n[1] = (ndim == 3) ? g->np[1] + 2 * nb : 1;
    g->n[2] = g->np[2] + 2 * nb;
    g->ncell = g->n[0] * g->n[1] * g->n[2];
    g->W = malloc(sizeof(double) * g->ncell);
    g->vc = malloc(sizeof(double) * g->ncell);
    g->ap = malloc(sizeof(double) * g->ncell);
    g->am = malloc(sizeof(double) * g->ncell);
    if (!g->W || !g->vc || !g->ap || !g->am) { og_free(g); return -3; }

    double vmax = 0.0;
    int64_t nphys = g->np[0] * g->np[1] * g->np[2];
    for (int64_t i = 0; i < nphys; ++i) if (v[i] > vmax) vmax = v[i];
    if (vref <= 0.0) vref = vmax;
    double emax[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < 3; ++a) {
        if (a == 1 && ndim == 2) continue;
        if (nb > 0) emax[a] = 3.0 * vref * log(1.0 / r0) / (2.0 * nb * h[a]);
    }
    int nby = (ndim == 3) ? nb : 0;
    for (int64_t iz = 0; iz < g->n[0]; ++iz)
        for (int64_t iy = 0; iy < g->n[1]; ++iy)
            for (int64_t ix = 0; ix < g->n[2]; ++ix) {
                int64_t pz = og_clamp(iz - nb, 0, g->np[0] - 1);
                int64_t py = og_clamp(iy - nby, 0, g->np[1] - 1);
                int64_t px = og_clamp(ix - nb, 0, g->np[2] - 1);
                double vv = v[(pz * g->np[1] + py) * g->np[2] + px];
                double eta = 0.0;
                if (nb > 0) {
                    double dz = og_depth(iz, g->np[0], nb) / nb;
                    double dx = og_depth(ix, g->np[2], nb) / nb;
                    eta += emax[0] * dz * dz + emax[2] * dx * dx;
                    if (ndim == 3) {
                        double dy = og_depth(iy, g->np[1], nb) / nb;
                        eta += emax[1] * dy * dy;
                    }
                }
                int64_t i = (iz * g->n[1] + iy) * g->n[2] + ix;
                g->vc[i] = vv;
                g->W[i] = vv * vv * dt * dt;
                g->ap[i] = 1.0 + eta * dt / 2.0;
                g->am[i] = 1.0 - eta * dt / 2.0;
            }
    return 0;
}

static int64_t og_index(const og_grid *g, const int32_t *p)
{
    int nby = (g->ndim == 3) ? g->nb : 0;
    int64_t iz = p[0] + g->nb, iy = p[1] + nby, ix = p[2] + g->nb;
    if (p[0] < 0 || p[0] >= g->np[0] || p[2] < 0 || p[2] >= g->np[2]) return -1;
    if (g->ndim == 3 && (p[1] < 0 || p[1] >= g->np[1])) return -1;
    if (g->ndim == 2 && p[1] != 0) return -1;
    return (iz * g->n[1] + iy) * g->n[2] + ix;
}

/* ------------------------------------------------------------------ points */

/* A source or receiver is a list of (node, weight) taps on the computed grid.  A grid
 * node is one tap of weight 1.  An off-grid position p (physical-grid index units,
 * fractional) uses Kaiser-windowed sinc interpolation (Hicks 2002): along each axis the
 * 2R nodes x nearest to p get
 *     w(x) = sinc(x - p) I0(b sqrt(1 - ((x - p) / R)^2)) / I0(b),
 * sinc(t) = sin(pi t) / (pi t), R = 4, b = 6.31, and a point takes the product of its
 * per-axis weights.  At an integer p the weights are 1 at p and 0 elsewhere (sinc
 * vanishes at the other integers), so a node given as a position is the node itself. */
#define OG_HW 4
#define OG_KB 6.31
#define OG_PI 3.14159265358979323846

typedef struct {
    int T;            /* taps per point */
    int64_t *idx;     /* [count][T] computed-grid cell indices */
    double *w;        /* [count][T] weights */
} og_pts;

/* modified Bessel function of the first kind, order 0: sum_k ((x/2)^k / k!)^2 */
static double og_i0(double x)
{
    double term = 1.0, sum = 1.0, q = 0.25 * x * x;
    for (int k = 1; k < 500; ++k) {
        term *= q / ((double)k * (double)k);
        sum += term;
        if (term < 1e-17 * sum) break;
    }
    return sum;
}

static double og_sinc(double t)
{
    if (t == floor(t)) return t == 0.0 ? 1.0 : 0.0;   /* sin(pi k) = 0 exactly */
    return sin(OG_PI * t) / (OG_PI * t);
}

/* weights of the 2R nodes first .. first + 2R - 1 along one axis for position p */
static void og_axis_weights(double p, int64_t *first, double *w)
{
    const int64_t i0 = (int64_t)floor(p);
    *first = i0 - OG_HW + 1;
    const double norm = og_i0(OG_KB);
    for (int k = 0; k < 2 * OG_HW; ++k) {
        const double t = (double)(*first + k) - p;
        const double r = t / OG_HW;
        const double win = fabs(r) <= 1.0 ? og_i0(OG_KB * sqrt(1.0 - r * r)) / norm : 0.0;
        w[k] = og_sinc(t) * win;
    }
}

static void og_pts_free(og_pts *p)
{
    free(p->idx);
    free(p->w);
    p->idx = NULL;
    p->w = NULL;
}

/* Taps of `count` points given as nodes (pos == NULL) or as positions ([count][3],
 * (z, y, x) physical-grid index units; y = 0 in 2-D).  Returns -1 when a node or a tap
 * falls outside its grid. */
static int og_points(const og_grid *g, int64_t count, const int32_t *nodes, const double *pos,
                     og_pts *out)
{
    const int two = 2 * OG_HW;
    out->T = pos ? (g->ndim == 3 ? two * two * two : two * two) : 1;
    const int64_t nalloc = (count > 0 ? count : 1) * out->T;
    out->idx = malloc(sizeof(int64_t) * nalloc);
    out->w = malloc(sizeof(double) * nalloc);
    if (!out->idx || !out->w) { og_pts_free(out); return -3; }
    const int nby = (g->ndim == 3) ? g->nb : 0;
    for (int64_t c = 0; c < count; ++c) {
        int64_t *ix = out->idx + c * out->T;
        double *wt = out->w + c * out->T;
        if (!pos) {
            ix[0] = og_index(g, nodes + 3 * c);
            wt[0] = 1.0;
            if (ix[0] < 0) return -1;
            continue;
        }
        const double *p = pos + 3 * c;
        if (!(p[0] >= 0.0 && p[0] <= (double)(g->np[0] - 1) && p[2] >= 0.0 &&
              p[2] <= (double)(g->np[2] - 1)))
            return -1;
        if (g->ndim == 3 && !(p[1] >= 0.0 && p[1] <= (double)(g->np[1] - 1))) return -1;
        if (g->ndim == 2 && p[1] != 0.0) return -1;
        int64_t fz, fy = 0, fx;
        double wz[2 * OG_HW], wy[2 * OG_HW], wx[2 * OG_HW];
        og_axis_weights(p[0] + g->nb, &fz, wz);
        og_axis_weights(p[2] + g->nb, &fx, wx);
        int ty = 1;
        if (g->ndim == 3) {
            og_axis_weights(p[1] + nby, &fy, wy);
            ty = two;
        } else {
            wy[0] = 1.0;
        }
        int t = 0;
        for (int a = 0; a < two; ++a)
            for (int b = 0; b < ty; ++b)
                for (int d = 0; d < two; ++d, ++t) {
                    const int64_t iz = fz + a, iy = fy + b, jx = fx + d;
                    if (iz < 0 || iz >= g->n[0] || iy < 0 || iy >= g->n[1] || jx < 0 ||
                        jx >= g->n[2])
                        return -1;
                    ix[t] = (iz * g->n[1] + iy) * g->n[2] + jx;
                    wt[t] = wz[a] * wy[b] * wx[d];
                }
    }
    return 0;
}

/* sum_t w_t u[idx_t] over the taps of point c */
static double og_sample(const og_pts *p, int64_t c, const double *u)
{
    double acc = 0.0;
    for (int t = 0; t < p->T; ++t) acc += p->w[c * p->T + t] * u[p->idx[c * p->T + t]];
    return acc;
}

/* u[idx_t] += w_t x over the taps of point c (the transpose of og_sample) */
static void og_spread(const og_pts *p, int64_t c, double x, double *u)
{
    for (int t = 0; t < p->T; ++t) u[p->idx[c * p->T + t]] += p->w[c * p->T + t] * x;
}

/* Taps of one point at position pos (physical-grid index units) on the computed grid of
 * the given shape and sponge width: writes up to (2R)^ndim cell indices and weights,
 * returns the tap count, or -1 outside the grid.  (For the interpolation pins.) */
int oracle_point_taps(int ndim, const int64_t *shape, int nb, const double *pos,
                      int64_t *idx, double *w)
{
    og_grid g;
    memset(&g, 0, sizeof(g));
    g.ndim = ndim;
    g.nb = nb;
    g.np[0] = shape[0];
    g.np[1] = ndim == 3 ? shape[1] : 1;
    g.np[2] = shape[2];
    g.n[0] = g.np[0] + 2 * nb;
    g.n[1] = ndim == 3 ? g.np[1] + 2 * nb : 1;
    g.n[2] = g.np[2] + 2 * nb;
    og_pts p;
    int rc = og_points(&g, 1, NULL, pos, &p);
    int T = p.T;
    if (rc == 0) {
        memcpy(idx, p.idx, sizeof(int64_t) * T);
        memcpy(w, p.w, sizeof(double) * T);
    }
    og_pts_free(&p);
    return rc == 0 ? T : -1;
}

/* ------------------------------------------------------------------ Laplacian */

static double og_at(const og_grid *g, const double *u, int64_t iz, int64_t iy, int64_t ix)
{
    if (iz < 0 || iz >= g->n[0] || iy < 0 || iy >= g->n[1] || ix < 0 || ix >= g->n[2])
        return 0.0;
    return u[(iz * g->n[1] + iy) * g->n[2] + ix];
}

/* L u = sum over axes a of (1/h_a^2) sum_{k=-M..M} c_|k| u(shifted k cells along a),
 * with u = 0 outside the computed grid (HRI Sec. 3: the Laplacian of Eq. 2-3 as a
 * central stencil of order 2M). */
static void og_laplacian(const og_grid *g, const double *u, double *out)
{
    const int M = g->M;
    const double *c = g->c;
    const double iz2 = 1.0 / (g->h[0] * g->h[0]);
    const double iy2 = 1.0 / (g->h[1] * g->h[1]);
    const double ix2 = 1.0 / (g->h[2] * g->h[2]);
    #pragma omp parallel for schedule(static)
    for (int64_t iz = 0; iz < g->n[0]; ++iz)
        for (int64_t iy = 0; iy < g->n[1]; ++iy)
            for (int64_t ix = 0; ix < g->n[2]; ++ix) {
                double u0 = og_at(g, u, iz, iy, ix);
                double sz = c[0] * u0, sx = c[0] * u0, sy = c[0] * u0;
                for (int k = 1; k <= M; ++k) {
                    sz += c[k] * (og_at(g, u, iz + k, iy, ix) + og_at(g, u, iz - k, iy, ix));
                    sx += c[k] * (og_at(g, u, iz, iy, ix + k) + og_at(g, u, iz, iy, ix - k));
                    if (g->ndim == 3)
                        sy += c[k] * (og_at(g, u, iz, iy + k, ix) + og_at(g, u, iz, iy - k, ix));
                }
                double lap = sz * iz2 + sx * ix2;
                if (g->ndim == 3) lap += sy * iy2;
                out[(iz * g->n[1] + iy) * g->n[2] + ix] = lap;
            }
}

/* The Laplacian alone, on a user grid with zero outside (no padding): for the tests of
 * convergence order and modified wavenumber. */
int oracle_laplacian(int ndim, const int64_t *shape, const double *h, int M,
                     const double *u, double *out)
{
    og_grid g;
    memset(&g, 0, sizeof(g));
    if (ndim != 2 && ndim != 3) return -1;
    if (oracle_fd_coeffs(M, g.c) != 0) return -1;
    g.ndim = ndim; g.M = M;
    for (int a = 0; a < 3; ++a) { g.n[a] = shape[a]; g.h[a] = h[a]; }
    if (ndim == 2) g.n[1] = 1;
    og_laplacian(&g, u, out);
    return 0;
}

/* ------------------------------------------------------------------ time stepping */

/* One damped leapfrog step (Eq. 3 with the sponge reading):
 *   a+ u^{n+1} = 2 u^n + W L u^n - a- u^{n-1} + dt^2 w[n] e_src
 * lap is scratch of the grid's size. */
/* a+ u^{n+1} = 2 u^n + W L u^n - a- u^{n-1} + dt^2 w[n] (source taps) */
static void og_step(const og_grid *g, const double *ucur, const double *uprev,
                    double *unext, double *lap, const og_pts *src, int64_t s, double srcval)
{
    og_laplacian(g, ucur, lap);
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < g->ncell; ++i)
        unext[i] = 2.0 * ucur[i] + g->W[i] * lap[i] - g->am[i] * uprev[i];
    og_spread(src, s, srcval, unext);
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < g->ncell; ++i) unext[i] /= g->ap[i];
}

typedef struct {
    int nshots, nrec, nt;
    const double *wavelet;  /* [nshots][nt] */
    og_pts src;             /* [nshots] points */
    og_pts rec;             /* [nshots][nrec] points */
} og_acq;

/* Source and receiver points from nodes (src, rec) or positions (src_pos, rec_pos) */
static int og_acq_build(const og_grid *g, og_acq *q, int nshots, const int32_t *src,
                        const double *src_pos, const double *wavelet, int nrec,
                        const int32_t *rec, const double *rec_pos, int nt)
{
    q->nshots = nshots;
    q->nrec = nrec;
    q->nt = nt;
    q->wavelet = wavelet;
    q->src.idx = q->rec.idx = NULL;
    q->src.w = q->rec.w = NULL;
    int rc = og_points(g, nshots, src, src_pos, &q->src);
    if (rc == 0) rc = og_points(g, (int64_t)nshots * nrec, rec, rec_pos, &q->rec);
    return rc;
}

static void og_acq_free(og_acq *q)
{
    og_pts_free(&q->src);
    og_pts_free(&q->rec);
}

/* Forward modelling of every shot.  traces[s][n][r] = u^{n+1}(rec_r).  final_u, when
 * given, receives per shot the last two states (u^nt, u^{nt-1}) on the computed grid. */
int oracle_forward(int ndim, const int64_t *shape, const double *h, const double *v,
                   double dt, int nt, int M, int nb, double r0, double vref,
                   int nshots, const int32_t *src, const double *src_pos,
                   const double *wavelet, int nrec, const int32_t *rec,
                   const double *rec_pos, double *traces, double *final_u)
{
    og_grid g;
    int rc = og_build(&g, ndim, shape, h, v, dt, M, nb, r0, vref);
    if (rc) return rc;
    og_acq q;
    rc = og_acq_build(&g, &q, nshots, src, src_pos, wavelet, nrec, rec, rec_pos, nt);
    double *a = calloc(g.ncell, sizeof(double));
    double *b = calloc(g.ncell, sizeof(double));
    double *c = calloc(g.ncell, sizeof(double));
    double *lap = malloc(sizeof(double) * g.ncell);
    if (rc) goto done;
    if (!a || !b || !c || !lap) { rc = -3; goto done; }
    for (int s = 0; s < nshots; ++s) {
        memset(a, 0, sizeof(double) * g.ncell);  /* u^{n-1} */
        memset(b, 0, sizeof(double) * g.ncell);  /* u^n */
        for (int n = 0; n < nt; ++n) {
            double w = wavelet[(int64_t)s * nt + n];
            og_step(&g, b, a, c, lap, &q.src, s, dt * dt * w);
            for (int r = 0; r < nrec; ++r)
                traces[((int64_t)s * nt + n) * nrec + r] =
                    og_sample(&q.rec, (int64_t)s * nrec + r, c);
            double *t = a; a = b; b = c; c = t;   /* (prev, cur) <- (cur, next) */
        }
        if (final_u) {
            memcpy(final_u + (2 * (int64_t)s) * g.ncell, b, sizeof(double) * g.ncell);
            memcpy(final_u + (2 * (int64_t)s + 1) * g.ncell, a, sizeof(double) * g.ncell);
        }
    }
done:
    free(a); free(b); free(c); free(lap);
    og_acq_free(&q);
    og_free(&g);
    return rc;
}

double oracle_misfit(const double *dmod, const double *dobs, int64_t n)
{
    double phi = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double r = dmod[i] - dobs[i];
        phi += r * r;   /* Eq. 1: squared L2 norm, no 1/2 and no dt weight */
    }
    return phi;
}

/* ------------------------------------------------------------------ adjoint */

/* Exact discrete adjoint of the damped leapfrog.  Derivation (Lagrangian of the
 * constraints a+ u^{m} - (2I + W L) u^{m-1} + a- u^{m-2} - dt^2 w[m-1] e_src = 0,
 * m = 1..nt): with nu^{nt+1} = nu^{nt+2} = 0, for m = nt down to 1,
 *   a+ nu^m = 2 nu^{m+1} + L (W nu^{m+1}) - a- nu^{m+2} + R^T q[m-1],
 * where q[n] is the trace-space adjoint source (2 (d - d_obs) for Eq. 1).  L is
 * symmetric and W diagonal, so the transposed step applies the stencil to W nu.
 * Then   d phi / d W = sum_{m=1}^{nt} nu^{m+1} (L u^m)   (zero-lag imaging) and the
 * wavelet sensitivity is  d / d w[n] = dt^2 nu^{n+1}(src).
 *
 * The forward history u^m, m = 1..nt-1, is needed in reverse order.  It is rebuilt
 * segment by segment from exact double-precision checkpoints (u^{a}, u^{a-1}) taken
 * every `seg` steps in a first forward sweep; recomputation repeats the same
 * arithmetic, so every u^m equals the stored-history value bit for bit. */
static int og_adjoint(const og_grid *g, const og_acq *q, int s, const double *adjsrc,
                      double *gW, double *xadj, int seg)
{
    const int nt = q->nt, nrec = q->nrec;
    const double dt = g->dt;
    if (seg < 1) seg = 1;
    int nseg = (nt + seg - 1) / seg;
    int rc = 0;
    double *ck = malloc(sizeof(double) * g->ncell * 2 * (size_t)nseg);
    double *hist = malloc(sizeof(double) * g->ncell * (size_t)(seg + 2));
    double *lap = malloc(sizeof(double) * g->ncell);
    double *tmp = malloc(sizeof(double) * g->ncell);
    double *n1 = calloc(g->ncell, sizeof(double));   /* nu^{m+1} */
    double *n2 = calloc(g->ncell, sizeof(double));   /* nu^{m+2} */
    double *n0 = calloc(g->ncell, sizeof(double));   /* nu^{m}   */
    double *ua = calloc(g->ncell, sizeof(double));
    double *ub = calloc(g->ncell, sizeof(double));
    double *uc = calloc(g->ncell, sizeof(double));
    if (!ck || !hist || !lap || !tmp || !n1 || !n2 || !n0 || !ua || !ub || !uc) {
        rc = -3; goto done;
    }
    const double *w = q->wavelet + (int64_t)s * nt;

    /* forward sweep: checkpoint (u^{k seg}, u^{k seg - 1}) for k = 0..nseg-1 */
    for (int n = 0; n < nt; ++n) {
        if (n % seg == 0) {
            int k = n / seg;
            memcpy(ck + (2 * (size_t)k) * g->ncell, ub, sizeof(double) * g->ncell);
            memcpy(ck + (2 * (size_t)k + 1) * g->ncell, ua, sizeof(double) * g->ncell);
        }
        og_step(g, ub, ua, uc, lap, &q->src, s, dt * dt * w[n]);
        double *t = ua; ua = ub; ub = uc; uc = t;
    }

    /* reverse sweep, one segment (a, a+seg] at a time, last segment first */
    int m = nt;
    for (int k = nseg - 1; k >= 0; --k) {
        int a = k * seg;
        int top = (a + seg < nt) ? a + seg : nt;
        /* rebuild u^{a}, ..., u^{top} into hist[0..top-a] */
        memcpy(hist, ck + (2 * (size_t)k) * g->ncell, sizeof(double) * g->ncell);
        memcpy(ua, ck + (2 * (size_t)k + 1) * g->ncell, sizeof(double) * g->ncell);
        for (int j = 1; j <= top - a; ++j) {
            const double *cur = hist + (size_t)(j - 1) * g->ncell;
            const double *prev = (j == 1) ? ua : hist + (size_t)(j - 2) * g->ncell;
            og_step(g, cur, prev, hist + (size_t)j * g->ncell, lap, &q->src, s,
                    dt * dt * w[a + j - 1]);
        }
        for (; m > a; --m) {
            /* nu^m from nu^{m+1}, nu^{m+2} and the adjoint source of sample m-1 */
            #pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < g->ncell; ++i) tmp[i] = g->W[i] * n1[i];
            og_laplacian(g, tmp, lap);
            #pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < g->ncell; ++i)
                n0[i] = 2.0 * n1[i] + lap[i] - g->am[i] * n2[i];
            const double *qm = adjsrc + ((int64_t)s * nt + (m - 1)) * nrec;
            for (int r = 0; r < nrec; ++r) og_spread(&q->rec, (int64_t)s * nrec + r, qm[r], n0);
            #pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < g->ncell; ++i) n0[i] /= g->ap[i];
            /* imaging: nu^{m+1} L u^m (nu^{nt+1} = 0 makes the m = nt term vanish) */
            if (m < nt && gW) {
                og_laplacian(g, hist + (size_t)(m - a) * g->ncell, lap);
                #pragma omp parallel for schedule(static)
                for (int64_t i = 0; i < g->ncell; ++i) gW[i] += n1[i] * lap[i];
            }
            if (xadj) xadj[(int64_t)s * nt + (m - 1)] = dt * dt * og_sample(&q->src, s, n0);
            double *t = n2; n2 = n1; n1 = n0; n0 = t;
        }
    }
done:
    free(ck); free(hist); free(lap); free(tmp);
    free(n1); free(n2); free(n0); free(ua); free(ub); free(uc);
    return rc;
}

/* Gradient of phi = sum_shots ||d_mod - d_obs||^2 with respect to the physical
 * velocity grid.  adjsrc, when given ([nshots][nt][nrec]), replaces 2 (d - d_obs) as
 * the adjoint source (then grad is J^T adjsrc, the Jacobian-transpose product, and
 * dobs is not read).  gW_out, when given, receives d phi / d W on the computed grid
 * (summed over shots).  seg is the checkpoint interval of the reverse sweep. */
int oracle_gradient(int ndim, const int64_t *shape, const double *h, const double *v,
                    double dt, int nt, int M, int nb, double r0, double vref,
                    int nshots, const int32_t *src, const double *src_pos,
                    const double *wavelet, int nrec, const int32_t *rec,
                    const double *rec_pos, const double *dobs, const double *adjsrc,
                    double *misfit, double *grad, double *gW_out, int seg)
{
    og_grid g;
    int rc = og_build(&g, ndim, shape, h, v, dt, M, nb, r0, vref);
    if (rc) return rc;
    og_acq q;
    rc = og_acq_build(&g, &q, nshots, src, src_pos, wavelet, nrec, rec, rec_pos, nt);
    int64_t ntr = (int64_t)nshots * nt * nrec;
    double *gW = calloc(g.ncell, sizeof(double));
    double *res = NULL;
    if (rc) goto done;
    if (!gW) { rc = -3; goto done; }
    if (!adjsrc) {
        double *dmod = malloc(sizeof(double) * (ntr > 0 ? ntr : 1));
        res = malloc(sizeof(double) * (ntr > 0 ? ntr : 1));
        if (!dmod || !res) { free(dmod); rc = -3; goto done; }
        rc = oracle_forward(ndim, shape, h, v, dt, nt, M, nb, r0, vref, nshots, src,
                            src_pos, wavelet, nrec, rec, rec_pos, dmod, NULL);
        if (rc) { free(dmod); goto done; }
        if (misfit) *misfit = oracle_misfit(dmod, dobs, ntr);
        for (int64_t i = 0; i < ntr; ++i) res[i] = 2.0 * (dmod[i] - dobs[i]);
        free(dmod);
        adjsrc = res;
    }
    for (int s = 0; s < nshots; ++s) {
        rc = og_adjoint(&g, &q, s, adjsrc, gW, NULL, seg);
        if (rc) goto done;
    }
    if (gW_out) memcpy(gW_out, gW, sizeof(double) * g.ncell);
    /* dW/dv_c = 2 v_c dt^2, then fold every computed cell onto the physical cell its
     * velocity was replicated from (the transpose of the edge-replication padding). */
    int64_t nphys = g.np[0] * g.np[1] * g.np[2];
    memset(grad, 0, sizeof(double) * nphys);
    int nby = (ndim == 3) ? nb : 0;
    for (int64_t iz = 0; iz < g.n[0]; ++iz)
        for (int64_t iy = 0; iy < g.n[1]; ++iy)
            for (int64_t ix = 0; ix < g.n[2]; ++ix) {
                int64_t i = (iz * g.n[1] + iy) * g.n[2] + ix;
                int64_t pz = og_clamp(iz - nb, 0, g.np[0] - 1);
                int64_t py = og_clamp(iy - nby, 0, g.np[1] - 1);
                int64_t px = og_clamp(ix - nb, 0, g.np[2] - 1);
                grad[(pz * g.np[1] + py) * g.np[2] + px] += 2.0 * g.vc[i] * dt * dt * gW[i];
            }
done:
    free(gW); free(res);
    og_acq_free(&q);
    og_free(&g);
    return rc;
}

/* Adjoint of the linear map wavelet -> traces (F: w -> d at fixed v):
 * x[s][n] = dt^2 nu^{n+1}(src_s), with y injected at the receivers. */
int oracle_source_adjoint(int ndim, const int64_t *shape, const double *h, const double *v,
                          double dt, int nt, int M, int nb, double r0, double vref,
                          int nshots, const int32_t *src, const double *src_pos, int nrec,
                          const int32_t *rec, const double *rec_pos, const double *y,
                          double *x)
{
    og_grid g;
    int rc = og_build(&g, ndim, shape, h, v, dt, M, nb, r0, vref);
    if (rc) return rc;
    double *zero = calloc((size_t)nshots * nt, sizeof(double));
    if (!zero) { og_free(&g); return -3; }
    og_acq q;
    rc = og_acq_build(&g, &q, nshots, src, src_pos, zero, nrec, rec, rec_pos, nt);
    for (int s = 0; s < nshots && rc == 0; ++s)
        rc = og_adjoint(&g, &q, s, y, NULL, x, nt);
    og_acq_free(&q);
    free(zero);
    og_free(&g);
    return rc;
}

/* Computed-grid extents and the W, a+ and a- fields the oracle uses (for the energy
 * test and for reports). */
int oracle_model_fields(int ndim, const int64_t *shape, const double *h, const double *v,
                        double dt, int M, int nb, double r0, double vref,
                        int64_t *ncomp, double *W, double *ap, double *am)
{
    og_grid g;
    int rc = og_build(&g, ndim, shape, h, v, dt, M, nb, r0, vref);
    if (rc) return rc;
    for (int a = 0; a < 3; ++a) ncomp[a] = g.n[a];
    if (W) memcpy(W, g.W, sizeof(double) * g.ncell);
    if (ap) memcpy(ap, g.ap, sizeof(double) * g.ncell);
    if (am) memcpy(am, g.am, sizeof(double) * g.ncell);
    og_free(&g);
    return 0;
}

/* ------------------------------------------------------------------ checkpoint codec */

/* Checkpoints of the reverse sweep (the paper only names the gradient, Sec. 1; the
 * checkpoint format is a reading): the state pair (u^n, u^{n-1}) is stored as the two
 * components a = u^n and d = u^n - u^{n-1} (single-precision difference), each as 16-bit
 * floats after scaling by its own s = 2^floor(log2(T / max|component|)), T = 2^14 for
 * IEEE half and T = 1 for bfloat16, with round-to-nearest-even; s = 1 for an all-zero
 * component and NaN when the pair holds a non-finite value; floor(log2 .) is clamped to
 * [-126, 127].  Decoding returns a and a - d.  Storing the difference keeps the part of
 * the state that drives the time stepping (u^n - u^{n-1}, about omega dt of u) to the
 * format's relative precision, instead of to that of u. */
float oracle_snap_scale(float maxabs, int dtype)
{
    if (dtype == 0 || maxabs == 0.0f) return 1.0f;
    if (!isfinite(maxabs)) return NAN;
    int texp = (dtype == 2) ? 14 : 0;
    int ex;
    double fr = frexp((double)maxabs, &ex);   /* maxabs = fr 2^ex, fr in [0.5, 1) */
    /* log2(T / max) = texp - ex - log2(fr), -log2(fr) in (0, 1] */
    int k = (fr == 0.5) ? texp - ex + 1 : texp - ex;
    if (k < -126) k = -126;
    if (k > 127) k = 127;
    return (float)ldexp(1.0, k);
}

static uint32_t or_bits(float f) { uint32_t x; memcpy(&x, &f, 4); return x; }
static float or_float(uint32_t x) { float f; memcpy(&f, &x, 4); return f; }

/* float -> bfloat16, round to nearest, ties to even (NaN stays a quiet NaN) */
uint16_t oracle_f32_to_bf16(float f)
{
    uint32_t x = or_bits(f);
    if ((x & 0x7fffffffu) > 0x7f800000u) return (uint16_t)((x >> 16) | 0x40u);
    uint32_t lsb = (x >> 16) & 1u;
    x += 0x7fffu + lsb;
    return (uint16_t)(x >> 16);
}

float oracle_bf16_to_f32(uint16_t h) { return or_float((uint32_t)h << 16); }

/* float -> IEEE binary16, round to nearest, ties to even, with subnormals, overflow to
 * infinity and NaN kept */
uint16_t oracle_f32_to_f16(float f)
{
    uint32_t x = or_bits(f);
    uint32_t sign = (x >> 16) & 0x8000u;
    uint32_t ax = x & 0x7fffffffu;
    if (ax >= 0x7f800000u) return (uint16_t)(sign | (ax > 0x7f800000u ? 0x7e00u : 0x7c00u));
    if (ax >= 0x477ff000u) return (uint16_t)(sign | 0x7c00u);   /* >= 65520: infinity */
    if (ax >= 0x38800000u) {                                     /* >= 2^-14: normal */
        uint32_t mant = ax & 0x7fffffu;
        uint32_t e = (ax >> 23) - 127u + 15u;
        uint32_t h = (e << 10) | (mant >> 13);
        uint32_t rem = mant & 0x1fffu;
        if (rem > 0x1000u || (rem == 0x1000u && (h & 1u))) h++;
        return (uint16_t)(sign | h);
    }
    if (ax < 0x33000000u) return (uint16_t)sign;                 /* < 2^-25: zero */
    /* subnormal result: count units of 2^-24 */
    uint32_t m = (ax & 0x7fffffu) | 0x800000u;
    int e = (int)(ax >> 23) - 127;                               /* -25 .. -15 */
    int shift = -e - 1;                                          /* 14 .. 24 */
    uint32_t q = m >> shift, rem = m & ((1u << shift) - 1u), half = 1u << (shift - 1);
    if (rem > half || (rem == half && (q & 1u))) q++;
    return (uint16_t)(sign | q);
}

float oracle_f16_to_f32(uint16_t h)
{
    uint32_t sign = ((uint32_t)h & 0x8000u) << 16;
    uint32_t e = (h >> 10) & 0x1fu, m = h & 0x3ffu;
    if (e == 0x1fu) return or_float(sign | 0x7f800000u | (m << 13));
    if (e == 0) return (sign ? -1.0f : 1.0f) * (float)ldexp((double)m, -24);
    return or_float(sign | ((e - 15u + 127u) << 23) | (m << 13));
}

/* Encode the pair (a, b) of n values: code[0..n) from a with scale[0], code[n..2n) from
 * d = a - b with scale[1]. */
void oracle_snap_encode(const float *a, const float *b, int64_t n, int dtype,
                        uint16_t *code, float *scale)
{
    float ma = 0.0f, md = 0.0f;
    int bad = 0;
    for (int64_t i = 0; i < n; ++i) {
        float d = a[i] - b[i];
        if (!isfinite(a[i]) || !isfinite(b[i])) bad = 1;
        if (fabsf(a[i]) > ma) ma = fabsf(a[i]);
        if (fabsf(d) > md) md = fabsf(d);
    }
    float sa = bad ? NAN : oracle_snap_scale(ma, dtype);
    float sd = bad ? NAN : oracle_snap_scale(md, dtype);
    scale[0] = sa;
    scale[1] = sd;
    for (int64_t i = 0; i < n; ++i) {
        float va = a[i] * sa;                 /* single-precision products, as stored */
        float vd = (a[i] - b[i]) * sd;
        code[i] = dtype == 2 ? oracle_f32_to_f16(va) : oracle_f32_to_bf16(va);
        code[n + i] = dtype == 2 ? oracle_f32_to_f16(vd) : oracle_f32_to_bf16(vd);
    }
}

void oracle_snap_decode(const uint16_t *code, const float *scale, int64_t n, int dtype,
                        float *a, float *b)
{
    for (int64_t i = 0; i < n; ++i) {
        float va = dtype == 2 ? oracle_f16_to_f32(code[i]) : oracle_bf16_to_f32(code[i]);
        float vd = dtype == 2 ? oracle_f16_to_f32(code[n + i]) : oracle_bf16_to_f32(code[n + i]);
        a[i] = va / scale[0];
        b[i] = a[i] - vd / scale[1];
    }
}
