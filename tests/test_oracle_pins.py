"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test below would fail for a plausible mistake in the oracle: a wrong coefficient
(moment conditions), a wrong index or axis in the stencil (modified-wavenumber symbol),
a wrong sign or a dropped term in the update (closed-box energy, Green's function), a
wrong time-order (self-convergence), a non-adjoint reverse sweep (dot-product tests) or
a wrong imaging condition / sponge fold (finite-difference gradients).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1912_08063_gb300 import synth


# ------------------------------------------------------------------ helpers

def exact_coeffs(M):
    """Symmetric second-derivative weights from the moment conditions
    sum_{k=-M..M} c_|k| k^(2j) = 2 [j == 1], j = 0..M, solved in exact rationals."""
    A = []
    b = []
    for j in range(M + 1):
        row = []
        for k in range(M + 1):
            if k == 0:
                row.append(Fraction(1 if j == 0 else 0))
            else:
                row.append(Fraction(2 * k ** (2 * j)))
        A.append(row)
        b.append(Fraction(2 if j == 1 else 0))
    n = M + 1
    for i in range(n):  # Gauss-Jordan on rationals
        p = next(r for r in range(i, n) if A[r][i] != 0)
        A[i], A[p] = A[p], A[i]
        b[i], b[p] = b[p], b[i]
        piv = A[i][i]
        A[i] = [a / piv for a in A[i]]
        b[i] = b[i] / piv
        for r in range(n):
            if r != i and A[r][i] != 0:
                f = A[r][i]
                A[r] = [a - f * c for a, c in zip(A[r], A[i])]
                b[r] = b[r] - f * b[i]
    return b


def symbol(M, theta):
    """1-D stencil symbol sum_k c_|k| e^{i k theta} (real) from the exact weights."""
    c = [float(x) for x in exact_coeffs(M)]
    return c[0] + 2.0 * sum(c[k] * math.cos(k * theta) for k in range(1, M + 1))


# ------------------------------------------------------------------ coefficients

@pytest.mark.parametrize("M", [1, 2, 4, 8])
def test_coefficients_match_exact_moment_solution(M):
    ex = exact_coeffs(M)
    c = oracle.fd_coeffs(M)
    for k in range(M + 1):
        assert abs(c[k] - float(ex[k])) <= 4e-16 * max(1.0, abs(float(ex[k]))), (k, c[k], ex[k])


def test_coefficients_8th_order_known_values():
    # Standard 8th-order central weights, written as rationals.
    assert exact_coeffs(4) == [Fraction(-205, 72), Fraction(8, 5), Fraction(-1, 5),
                               Fraction(8, 315), Fraction(-1, 560)]


# ------------------------------------------------------------------ Laplacian

@pytest.mark.parametrize("ndim,M", [(2, 4), (3, 4), (2, 8), (3, 8)])
def test_laplacian_modified_wavenumber(ndim, M):
    """L cos(k.x + phase) = sum_a symbol(k_a h_a) / h_a^2 cos(...) exactly away from
    the edges (trig identity), for anisotropic spacing and wavenumbers per axis."""
    rng = np.random.default_rng(7)
    if ndim == 2:
        shape, h = (40, 44), (7.0, 1.0, 11.0)
        axes = [0, 2]
    else:
        shape, h = (36, 38, 40), (7.0, 9.0, 11.0)
        axes = [0, 1, 2]
    k = rng.uniform(0.2, 2.8, 3) / np.array(h)
    ph = rng.uniform(0, 2 * np.pi, 3)
    grids = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    if ndim == 2:
        coords = {0: grids[0], 2: grids[1]}
    else:
        coords = {0: grids[0], 1: grids[1], 2: grids[2]}
    u = np.ones(shape)
    for a in axes:
        u = u * np.cos(k[a] * h[a] * coords[a] + ph[a])
    lap = oracle.laplacian(u, h, M)
    expect_factor = sum(symbol(M, k[a] * h[a]) / h[a] ** 2 for a in axes)
    sl = tuple(slice(M, n - M) for n in shape)
    err = np.abs(lap[sl] - expect_factor * u[sl]).max()
    assert err <= 1e-12 * abs(expect_factor), err


@pytest.mark.parametrize("M,lo,hi,hset", [(4, 7.5, 8.5, (0.55, 0.45, 0.35, 0.28)),
                                          (8, 15.0, 17.0, (0.62, 0.55, 0.47, 0.4))])
def test_laplacian_convergence_order(M, lo, hi, hset):
    """Error of L on sin(az) sin(bx) against the exact -(a^2+b^2) f falls as h^(2M)
    (h ranges chosen above the FP64 round-off floor)."""
    a, b = 1.3, 0.9
    errs, hs = [], []
    for h in hset:
        n = int(round(40.0 / h))
        z = np.arange(n) * h
        f = np.sin(a * z)[:, None] * np.sin(b * z)[None, :]
        lap = oracle.laplacian(f, (h, 1.0, h), M)
        m = slice(M, n - M)
        err = np.abs(lap[m, m] + (a * a + b * b) * f[m, m]).max()
        errs.append(err)
        hs.append(h)
    slope = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    assert lo <= slope <= hi, (slope, errs)


@pytest.mark.parametrize("M", [4, 8])
def test_cfl_number_matches_stencil_eigenvalue(M):
    """The stability number uses the largest eigenvalue of the periodic 1-D stencil,
    found here numerically from the circulant matrix."""
    c = oracle.fd_coeffs(M)
    n = 64
    A = np.zeros((n, n))
    for i in range(n):
        A[i, i] = c[0]
        for k in range(1, M + 1):
            A[i, (i + k) % n] += c[k]
            A[i, (i - k) % n] += c[k]
    S = np.abs(np.linalg.eigvalsh(A)).max()
    h = (10.0, 12.0, 15.0)
    for ndim in (2, 3):
        acc = S / h[0] ** 2 + S / h[2] ** 2 + (S / h[1] ** 2 if ndim == 3 else 0.0)
        expect = 3000.0 * 1e-3 * math.sqrt(acc) / 2.0
        got = oracle.cfl_number(ndim, M, h, 3000.0, 1e-3)
        assert abs(got - expect) <= 1e-10 * expect


def _closed_box(ndim, M, nt, courant_scale, seed=3, noise=False, homogeneous=False):
    rng = np.random.default_rng(seed)
    shape = (24, 26) if ndim == 2 else (14, 15, 16)
    h = 10.0
    v = rng.uniform(1800.0, 3000.0, shape)
    if homogeneous:
        v[...] = 2500.0
    lim_dt = 1.0 / oracle.cfl_number(ndim, M, (h, h, h), v.max(), 1.0)
    dt = courant_scale * lim_dt
    src = [[shape[0] // 2, 0 if ndim == 2 else shape[1] // 2, shape[-1] // 3]]
    rec = [[2, 0 if ndim == 2 else 3, 4]]
    if noise:
        w = rng.standard_normal(nt)
    else:
        w = np.zeros(nt)
        w[:6] = rng.standard_normal(6)
    return oracle.Problem(v, h, dt, nt, order=2 * M, nb=0, src=src, rec=rec, wavelet=w)


@pytest.mark.parametrize("ndim,M", [(2, 4), (3, 4), (2, 8), (3, 8)])
def test_closed_box_energy_is_conserved(ndim, M):
    """With no sponge and zero Dirichlet walls, E = |u^{n+1}-u^n|^2_{1/W} - <u^{n+1}, L u^n>
    is constant once the source is silent (discrete energy of the leapfrog)."""
    energies = []
    for nt in (10, 40, 90):
        p = _closed_box(ndim, M, nt, 0.8)
        _, fin = p.forward(final=True)
        W, _, _ = p.fields()
        un1, un = fin[0, 0], fin[0, 1]
        lap = oracle.laplacian(un, p.h, p.M)
        E = np.sum((un1 - un) ** 2 / W) - np.sum(un1 * lap)
        energies.append(E)
    e0 = energies[0]
    assert e0 > 0
    for e in energies[1:]:
        assert abs(e - e0) <= 1e-11 * abs(e0), energies


def test_sponge_dissipates_energy():
    rng = np.random.default_rng(5)
    shape = (30, 32)
    v = rng.uniform(1800.0, 2600.0, shape)
    w = np.zeros(500)
    w[:5] = 1.0
    es = []
    for nt in (20, 60, 120, 250, 500):
        p = oracle.Problem(v, 10.0, 1e-3, nt, order=8, nb=10, src=[[15, 0, 16]],
                           rec=[[3, 0, 3]], wavelet=w[:nt])
        _, fin = p.forward(final=True)
        W, ap, am = p.fields()
        un1, un = fin[0, 0], fin[0, 1]
        lap = oracle.laplacian(un, p.h, p.M)
        es.append(np.sum((un1 - un) ** 2 / W) - np.sum(un1 * lap))
    assert all(b < a for a, b in zip(es, es[1:])), es
    assert es[-1] < 0.2 * es[0]


def test_sponge_reflection_is_small():
    """A trace recorded near the sponge of a small homogeneous box matches the same trace
    in a box large enough that nothing comes back within the window: the sponge's
    reflection stays below 2 % of the direct wave."""
    c, h, dt, nt, f0 = 2000.0, 10.0, 1e-3, 300, 12.0
    w = synth.ricker(f0, dt, nt).astype(np.float64)
    traces = []
    for n in (61, 241):
        o = (n - 61) // 2
        p = oracle.Problem(np.full((n, n), c), h, dt, nt, order=8, nb=20,
                           src=[[30 + o, 0, 30 + o]], rec=[[30 + o, 0, 52 + o]], wavelet=w)
        traces.append(p.forward()[0, :, 0])
    err = np.linalg.norm(traces[0] - traces[1]) / np.linalg.norm(traces[1])
    assert err < 2e-2, err


def test_cfl_boundary_is_the_stability_boundary():
    """In a homogeneous closed box, below the stability number the run stays bounded;
    10 % above it the highest (checkerboard) mode grows without bound."""
    for M in (4, 8):
        ok = _closed_box(2, M, 400, 0.97, noise=True, homogeneous=True).forward()
        bad = _closed_box(2, M, 400, 1.10, noise=True, homogeneous=True).forward()
        assert np.all(np.isfinite(ok)) and np.abs(ok).max() < 1e3
        assert not np.all(np.isfinite(bad)) or np.abs(bad).max() > 1e20


# ------------------------------------------------------------------ physics

def _green_3d(w, dt, nt, r, c, h):
    t = (np.arange(nt) + 1) * dt - r / c
    f0, t0 = w
    a = (np.pi * f0 * (t - t0)) ** 2
    wv = (1 - 2 * a) * np.exp(-a)
    return h ** 3 * wv / (4 * np.pi * c * c * r)


def _green_2d(w, dt, nt, r, c, h):
    f0, t0 = w
    th = np.linspace(0.0, 12.0, 24001)
    out = np.zeros(nt)
    for n in range(nt):
        t = (n + 1) * dt
        tau = t - (r / c) * np.cosh(th)
        a = (np.pi * f0 * (tau - t0)) ** 2
        out[n] = np.trapezoid((1 - 2 * a) * np.exp(-a), th)
    return h ** 2 * out / (2 * np.pi * c * c)


@pytest.mark.parametrize("ndim", [2, 3])
def test_homogeneous_greens_function(ndim):
    """A point source in a homogeneous medium: the trace at distance r matches the
    free-space Green's function convolved with the Ricker wavelet, for the node
    injection dt^2 w[n] (a source density h^d w(t) delta(x))."""
    c, h, dt = 2000.0, 10.0, 1e-3
    f0 = 8.0
    if ndim == 2:
        n, nt = 81, 380
        shape = (n, n)
        src = [[40, 0, 40]]
        rec = [[40, 0, 52], [28, 0, 40], [52, 0, 55]]
    else:
        n, nt = 49, 300
        shape = (n, n, n)
        src = [[24, 24, 24]]
        rec = [[24, 24, 36], [12, 24, 24], [30, 30, 33]]
    v = np.full(shape, c)
    w = synth.ricker(f0, dt, nt).astype(np.float64)
    p = oracle.Problem(v, h, dt, nt, order=8, nb=20, src=src, rec=rec, wavelet=w)
    tr = p.forward()[0]
    for j, rr in enumerate(rec):
        r = h * math.sqrt(sum((a - b) ** 2 for a, b in zip(rr, src[0])))
        g = (_green_2d if ndim == 2 else _green_3d)((f0, 1.5 / f0), dt, nt, r, c, h)
        err = np.linalg.norm(tr[:, j] - g) / np.linalg.norm(g)
        assert err < 0.03, (j, err)


def test_time_stepping_is_second_order():
    """Self-convergence under dt -> dt/2 -> dt/4 on a fixed grid: successive trace
    differences shrink by about 4."""
    c, h = 2000.0, 10.0
    shape = (61, 61)
    v = np.full(shape, c)
    v[35:, :] = 2600.0
    T = 0.24
    outs = []
    for dt in (1.6e-3, 0.8e-3, 0.4e-3):
        nt = int(round(T / dt))
        w = synth.ricker(10.0, dt, nt).astype(np.float64)
        p = oracle.Problem(v, h, dt, nt, order=8, nb=10, src=[[20, 0, 30]],
                           rec=[[20, 0, 42], [40, 0, 30]], wavelet=w)
        tr = p.forward()[0]
        # common sample times t = k * 1.6 ms
        step = int(round(1.6e-3 / dt))
        outs.append(tr[step - 1::step][: int(round(T / 1.6e-3))])
    d1 = np.linalg.norm(outs[0] - outs[1])
    d2 = np.linalg.norm(outs[1] - outs[2])
    ratio = d1 / d2
    assert 3.4 < ratio < 4.6, ratio


# ------------------------------------------------------------------ adjoint

def _hetero_problem(ndim, M, nt=50, nb=6, seed=11, nrec=5, dup=True):
    rng = np.random.default_rng(seed)
    shape = (18, 21) if ndim == 2 else (11, 12, 13)
    h = 10.0
    v = rng.uniform(1600.0, 3200.0, shape)
    dt = 0.5 / oracle.cfl_number(ndim, M, (h, h, h), v.max(), 1.0)
    if ndim == 2:
        src = [[3, 0, 7], [10, 0, 2]]
        rec = np.stack([rng.integers(0, shape[0], nrec), np.zeros(nrec, int),
                        rng.integers(0, shape[1], nrec)], 1)
    else:
        src = [[3, 4, 7], [7, 1, 2]]
        rec = np.stack([rng.integers(0, s, nrec) for s in shape], 1)
    if dup:
        rec[1] = rec[0]
    w = rng.standard_normal((2, nt))
    return oracle.Problem(v, h, dt, nt, order=2 * M, nb=nb, vref=3500.0, src=src,
                          rec=rec, wavelet=w), rng


@pytest.mark.parametrize("ndim,M", [(2, 4), (3, 4), (2, 8), (3, 8)])
def test_source_dot_product(ndim, M):
    """<F x, y> = <x, F* y> for the linear map wavelet -> traces, sponge on."""
    p, rng = _hetero_problem(ndim, M)
    x = rng.standard_normal((p.nshots, p.nt))
    y = rng.standard_normal((p.nshots, p.nt, p.nrec))
    Fx = p.forward(wavelet=x)
    Fty = p.source_adjoint(y)
    lhs, rhs = np.sum(Fx * y), np.sum(x * Fty)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs)), (lhs, rhs)


@pytest.mark.parametrize("ndim,M", [(2, 4), (3, 8)])
def test_jacobian_dot_product(ndim, M):
    """<J dv, y> (central difference of the forward map) = <dv, J^T y> (reverse sweep
    with y as adjoint source)."""
    p, rng = _hetero_problem(ndim, M, nt=40)
    y = rng.standard_normal((p.nshots, p.nt, p.nrec))
    dv = rng.standard_normal(p.v.shape) * 10.0
    _, JTy = p.gradient(adjsrc=y, seg=7)
    eps = 1e-3
    Jdv = (p.forward(v=p.v + eps * dv) - p.forward(v=p.v - eps * dv)) / (2 * eps)
    lhs, rhs = np.sum(Jdv * y), np.sum(dv * JTy)
    assert abs(lhs - rhs) <= 1e-7 * abs(rhs), (lhs, rhs)


def _fd_case(ndim):
    if ndim == 2:
        shape = (40, 40)
        nt, h = 140, 10.0
    else:
        shape = (24, 24, 24)
        nt, h = 70, 10.0
    rng = np.random.default_rng(21)
    v = synth.smooth_random(rng, shape, h, ell=80.0)
    vobs = v * (1.0 + 0.03 * synth.gaussian_random_field(rng, shape, h, 60.0, 1.0))
    dt = 0.45 / oracle.cfl_number(ndim, 4, (h, h, h), 4800.0, 1.0)
    if ndim == 2:
        src = [[5, 0, 20]]
        rec = [[3, 0, i] for i in range(0, 40, 3)]
    else:
        src = [[5, 12, 12]]
        rec = [[3, j, i] for j in range(0, 24, 5) for i in range(0, 24, 5)]
    w = synth.ricker(40.0, dt, nt).astype(np.float64)
    mk = lambda vv: oracle.Problem(vv, h, dt, nt, order=8, nb=8, vref=4800.0, src=src,
                                   rec=rec, wavelet=w)
    dobs = mk(vobs).forward()
    return mk(v), dobs, rng


@pytest.mark.parametrize("ndim", [2, 3])
def test_gradient_directional_finite_difference(ndim):
    p, dobs, rng = _fd_case(ndim)
    phi, g = p.gradient(dobs)
    dv = synth.gaussian_random_field(rng, p.v.shape, 10.0, 60.0, 1.0).astype(np.float64)
    dv *= 50.0
    eps = 1e-4  # the central difference's own error is O(eps^2): ~1e-8 relative here
    fp = oracle.misfit(p.forward(v=p.v + eps * dv), dobs)
    fm = oracle.misfit(p.forward(v=p.v - eps * dv), dobs)
    fd = (fp - fm) / (2 * eps)
    an = np.sum(g * dv)
    assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)
    assert phi > 0


def test_gradient_pointwise_including_sponge_edge():
    """Point-wise central differences at interior cells and at an edge cell whose
    velocity is replicated into the sponge (checks the fold of sponge cells)."""
    p, dobs, _ = _fd_case(2)
    _, g = p.gradient(dobs)
    cells = [(20, 20), (6, 21), (30, 10), (39, 17), (12, 0)]
    for (iz, ix) in cells:
        eps = 0.5
        vp, vm = p.v.copy(), p.v.copy()
        vp[iz, ix] += eps
        vm[iz, ix] -= eps
        fd = (oracle.misfit(p.forward(v=vp), dobs) - oracle.misfit(p.forward(v=vm), dobs)) / (2 * eps)
        assert abs(fd - g[iz, ix]) <= 1e-5 * np.abs(g).max(), ((iz, ix), fd, g[iz, ix])


def test_gradient_checkpoint_interval_does_not_change_result():
    p, dobs, _ = _fd_case(2)
    a = p.gradient(dobs, seg=1)[1]
    b = p.gradient(dobs, seg=13)[1]
    c = p.gradient(dobs, seg=p.nt)[1]
    assert np.array_equal(a, b) and np.array_equal(a, c)
