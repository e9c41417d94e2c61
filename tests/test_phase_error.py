"""Phase-error study of the 8th- and 16th-order stencils (the experiment of Sec. 4,
Fig. 6: the second derivative of a cosine versus stencil order and sampling).

The oracle's Laplacian is applied to cos(k x) sampled at N points per wavelength; the
ratio of the result to the exact -k^2 cos(k x) gives the relative error of the second
derivative, and its square root the relative phase-velocity error of the semi-discrete
wave equation.  For a tolerance, the coarsest sampling each order allows gives the
per-axis domain saving of 16th over 8th order.  The paper prints "12 %"; with Taylor
weights the saving is larger at every tolerance tighter than about 5 % phase-velocity
error (the figure's data are not in the text, so the 12 % is not pinned)."""
import math

import numpy as np
import pytest

import oracle
from test_oracle_pins import symbol


def phase_error(M, ppw):
    """Relative phase-velocity error at `ppw` points per wavelength, measured by applying
    the oracle's Laplacian to a sampled cosine (interior points of a 2-D grid)."""
    h = 1.0
    k = 2 * math.pi / (ppw * h)
    nx = 64
    x = np.arange(nx) * h
    u = np.ones((2 * M + 3, 1)) * np.cos(k * x + 0.3)[None, :]
    lap = oracle.laplacian(u, (1e9, 1.0, h), M)     # z spacing huge: x-derivative alone
    sl = (M + 1, slice(M, nx - M))
    ratio = lap[sl] / (-(k * k) * u[sl])
    return abs(math.sqrt(float(np.mean(ratio))) - 1.0)


def coarsest_sampling(M, tol):
    lo, hi = 2.01, 200.0
    for _ in range(60):   # phase error decreases with ppw: bisect the threshold
        mid = 0.5 * (lo + hi)
        if phase_error(M, mid) <= tol:
            hi = mid
        else:
            lo = mid
    return hi


@pytest.mark.parametrize("M", [4, 8])
def test_phase_error_matches_closed_form(M):
    for ppw in (3.0, 4.0, 6.0, 10.0):
        k = 2 * math.pi / ppw
        closed = abs(math.sqrt(-symbol(M, k) / (k * k)) - 1.0)
        assert abs(phase_error(M, ppw) - closed) <= 1e-9


def test_domain_saving_sixteenth_over_eighth_order():
    rows = []
    for tol in (5e-2, 1e-2, 1e-3, 1e-4, 1e-5, 1e-6):
        n8, n16 = coarsest_sampling(4, tol), coarsest_sampling(8, tol)
        rows.append((tol, n8, n16, 1.0 - n16 / n8))
    for tol, n8, n16, s in rows:
        print(f"tol {tol:.0e}: {n8:6.2f} vs {n16:6.2f} points per wavelength, saving {100 * s:5.1f} %")
    savings = [s for *_, s in rows]
    assert all(b > a for a, b in zip(savings, savings[1:]))   # grows as the tolerance tightens
    assert 0.05 < savings[0] < 0.2                           # about the paper's 12 % near 5 %
    assert 0.2 < savings[1] and savings[-1] < 0.6
