"""The transposed form of the zero-lag imaging sum that the GPU reverse step uses.

For the damped leapfrog  a+ u^{n+1} = 2 u^n + W L u^n - a- u^{n-1} + F^n  (u^0 = u^-1 = 0)
and its adjoint in mu = W nu,
a+ mu^m = 2 mu^{m+1} + W L mu^{m+1} - a- mu^{m+2} + a+ J^m  (mu^{nt+1} = mu^{nt+2} = 0),
the imaging sum of the textbook adjoint-state gradient satisfies, point by point,

  sum_{m=0}^{nt-1} mu^{m+1} L u^m
      = sum_{m=1}^{nt-1} u^m L mu^{m+1}  +  sum_{m=1}^{nt} u^m (a+ / W) J^m
        - sum_{m=0}^{nt-1} mu^{m+1} F^m / W.

It follows from substituting the forward recursion for W L u^m, re-indexing the sum over
time and substituting the adjoint recursion; L need not be symmetric.  With J^m the
receiver injection 2 W / a+ r^{m-1} the middle term is 2 sum_k d^k r^k at each receiver.
This test runs both recursions in FP64 (the oracle's Laplacian) and checks the identity
to rounding, including coincident source and receiver nodes and a receiver in the sponge.
"""
import numpy as np
import pytest

import oracle


def _run(seed, M, nz=18, nx=22, nt=40, src=(9, 11), recs=((3, 4), (3, 15), (9, 11), (16, 2))):
    rng = np.random.default_rng(seed)
    h = (7.0, 9.0)
    W = rng.uniform(0.02, 0.08, (nz, nx))                # v^2 dt^2 (stable for these h)
    sig = np.zeros((nz, nx))
    sig[:3, :] += 0.05
    sig[:, -3:] += 0.08                                   # a sponge strip on two sides
    ap, am = 1.0 + sig, 1.0 - sig
    w = rng.standard_normal(nt)                           # wavelet samples
    dobs = rng.standard_normal((nt, len(recs)))
    L = lambda f: oracle.laplacian(f, h, M)

    u = [np.zeros((nz, nx)) for _ in range(nt + 1)]      # u^0 .. u^nt
    prev = np.zeros((nz, nx))
    for n in range(nt):
        F = np.zeros((nz, nx))
        F[src] = w[n]
        nxt = (2 * u[n] + W * L(u[n]) - am * prev + F) / ap
        prev = u[n]
        u[n + 1] = nxt
    d = np.array([[u[k + 1][r] for r in recs] for k in range(nt)])
    res = d - dobs

    inj = 2.0 * W / ap
    mu = {nt + 1: np.zeros((nz, nx)), nt + 2: np.zeros((nz, nx))}
    Jm = {}
    for m in range(nt, 0, -1):
        J = np.zeros((nz, nx))
        for i, r in enumerate(recs):
            J[r] += inj[r] * res[m - 1, i]
        Jm[m] = J
        mu[m] = (2 * mu[m + 1] + W * L(mu[m + 1]) - am * mu[m + 2]) / ap + J

    g_text = sum(mu[m + 1] * L(u[m]) for m in range(nt))
    g_tr = sum(u[m] * L(mu[m + 1]) for m in range(1, nt))
    g_tr = g_tr + sum(u[m] * ap / W * Jm[m] for m in range(1, nt + 1))
    Fsum = np.zeros((nz, nx))
    Fsum[src] = sum(w[m] * mu[m + 1][src] for m in range(nt))
    g_tr = g_tr - Fsum / W
    # the receiver term written from the traces alone, as the library adds it
    rec_term = np.zeros((nz, nx))
    for i, r in enumerate(recs):
        rec_term[r] += 2.0 * np.sum(d[:, i] * res[:, i])
    rec_direct = sum(u[m] * ap / W * Jm[m] for m in range(1, nt + 1))
    return g_text, g_tr, rec_term, rec_direct


@pytest.mark.parametrize("M", [4, 8])
def test_transposed_imaging_identity(M):
    g_text, g_tr, rec_term, rec_direct = _run(1 + M, M)
    scale = np.abs(g_text).max()
    assert scale > 0
    assert np.abs(g_tr - g_text).max() <= 1e-10 * scale
    assert np.abs(rec_term - rec_direct).max() <= 1e-10 * np.abs(rec_direct).max()


def test_identity_fails_without_the_point_terms():
    """The point terms are needed: leaving out either one breaks the identity where the
    source or a receiver sits (a guard against a test that passes vacuously)."""
    g_text, g_tr, rec_term, _ = _run(3, 4)
    bad = g_tr - rec_term
    assert np.abs(bad - g_text).max() > 1e-3 * np.abs(g_text).max()
