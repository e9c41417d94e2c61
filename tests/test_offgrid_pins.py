"""Pins of the oracle's off-grid sources and receivers (Kaiser-windowed sinc points,
Hicks 2002: half-width 4, b = 6.31), checked against what the mathematics fixes:

* a position on a node is that node (the weights are a delta);
* the weights interpolate band-limited fields: sampled cosines of wavelength >= 4
  cells are reproduced at arbitrary positions to ~1e-3 (the windowed sinc's design
  accuracy), far better than the nearest node;
* injection is the transpose of sampling: the dot-product test of the wavelet-to-trace
  map holds to rounding with off-grid sources and receivers;
* the gradient with off-grid points matches central finite differences.
"""
import numpy as np
import pytest

import oracle
from paper_1912_08063_gb300 import synth


def _cos_field(shape, nb, k, theta, phi, psi):
    """cos(k . x + psi) on the computed grid (index units) for a wave vector of modulus
    k and direction (theta, phi)."""
    n = [s + 2 * nb for s in shape]
    if len(shape) == 2:
        kv = k * np.array([np.cos(theta), np.sin(theta)])
    else:
        kv = k * np.array([np.cos(theta), np.sin(theta) * np.cos(phi),
                           np.sin(theta) * np.sin(phi)])
    grids = np.meshgrid(*[np.arange(m) for m in n], indexing="ij")
    return np.cos(sum(kk * g for kk, g in zip(kv, grids)) + psi), kv


@pytest.mark.parametrize("shape", [(30, 40), (22, 18, 26)])
def test_weights_interpolate_sampled_cosines(shape):
    rng = np.random.default_rng(len(shape))
    nb = 20
    tol = 2e-3 if len(shape) == 2 else 3e-3
    worst_near = 0.0
    for lam in (4.0, 6.0, 10.0):
        for _ in range(12):
            theta, phi, psi = rng.uniform(0, 2 * np.pi, 3)
            u, kv = _cos_field(shape, nb, 2 * np.pi / lam, theta, phi, psi)
            p = np.array([rng.uniform(0, s - 1) for s in shape])
            idx, w = oracle.point_taps(shape, p, nb)
            val = float(np.dot(w, u.ravel()[idx]))
            ref = float(np.cos(np.dot(kv, p + nb) + psi))
            assert abs(val - ref) < tol, (lam, p, val, ref)
            near = u[tuple(np.rint(p + nb).astype(int))]
            worst_near = max(worst_near, abs(near - ref))
    assert worst_near > 10 * tol   # the nearest node is much worse: the test has teeth


def test_node_position_is_the_node():
    """Sources and receivers given as integer positions reproduce the node-based run
    bit for bit."""
    w = synth.random_small(np.random.default_rng(4), 2, (24, 30), nt=60, nb=20)
    P_nodes = oracle.Problem(w.v, w.h, w.dt, w.nt, order=8, nb=20, src=w.src, rec=w.rec,
                             wavelet=w.wavelets())
    P_pos = oracle.Problem(w.v, w.h, w.dt, w.nt, order=8, nb=20,
                           src_pos=np.asarray(w.src, dtype=np.float64),
                           rec_pos=np.asarray(w.rec, dtype=np.float64), wavelet=w.wavelets())
    assert np.array_equal(P_nodes.forward(), P_pos.forward())


def _offgrid_problem(ndim, seed=7):
    rng = np.random.default_rng(seed)
    shape = (20, 26) if ndim == 2 else (14, 12, 16)
    v = 2000.0 + 300.0 * rng.random(shape)
    h = (10.0,) * ndim
    dt, nt = 1e-3, 50 if ndim == 2 else 36
    nshots, nrec = 2, 5
    src_pos = np.stack([np.array([rng.uniform(1, s - 2) if (ndim == 3 or a != 1) else 0.0
                                  for a, s in enumerate((shape[0], 1 if ndim == 2 else shape[1], shape[-1]))])
                        for _ in range(nshots)])
    rec_pos = np.stack([[np.array([rng.uniform(1, s - 2) if (ndim == 3 or a != 1) else 0.0
                                   for a, s in enumerate((shape[0], 1 if ndim == 2 else shape[1], shape[-1]))])
                         for _ in range(nrec)] for _ in range(nshots)])
    wav = np.stack([synth.ricker(25.0, dt, nt) * (1 + 0.2 * s) for s in range(nshots)])
    # sponge reference velocity fixed, so the sponge does not move with v
    P = oracle.Problem(v, h, dt, nt, order=8, nb=20, vref=3000.0, src_pos=src_pos,
                       rec_pos=rec_pos, wavelet=wav)
    return P, v, rng


@pytest.mark.parametrize("ndim", [2, 3])
def test_offgrid_source_dot_product(ndim):
    """<F x, y> = <x, F* y> for the wavelet-to-trace map with off-grid points: sampling
    and injection use the same weights, transposed."""
    P, v, rng = _offgrid_problem(ndim)
    x = rng.standard_normal((P.nshots, P.nt))
    y = rng.standard_normal((P.nshots, P.nt, P.nrec))
    Fx = P.forward(wavelet=x)
    Fty = P.source_adjoint(y)
    lhs, rhs = float(np.sum(Fx * y)), float(np.sum(x * Fty))
    assert abs(lhs - rhs) <= 1e-11 * max(abs(lhs), abs(rhs))


def test_offgrid_gradient_matches_finite_differences():
    P, v, rng = _offgrid_problem(2, seed=11)
    dobs = P.forward(v=v * (1.0 + 0.03 * rng.standard_normal(v.shape)))
    phi0, g = P.gradient(dobs)
    dv = rng.standard_normal(v.shape)
    eps = 1e-3
    fp = P.gradient(dobs, v=v + eps * dv)[0]
    fm = P.gradient(dobs, v=v - eps * dv)[0]
    fd = (fp - fm) / (2 * eps)
    an = float(np.sum(g * dv))
    assert abs(fd - an) <= 1e-7 * abs(an)
