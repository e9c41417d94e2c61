"""CPU-only checks of the C-ABI library: it loads, exports every declared symbol, and its
host logic (stencil weights, stability number, checkpoint schedule) is right.  No call
here touches a GPU."""
import os
import re
from functools import lru_cache

import numpy as np
import pytest

import oracle
from paper_1912_08063_gb300 import fwi
from test_oracle_pins import exact_coeffs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "fwi.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fwi_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    L = fwi.lib()
    names = declared_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n


@pytest.mark.parametrize("order", [8, 16])
def test_host_coefficients_are_exact(order):
    c = fwi.fwi_fd_coeffs(order)
    ex = exact_coeffs(order // 2)
    for k, e in enumerate(ex):
        assert abs(c[k] - float(e)) <= 4e-16 * max(1.0, abs(float(e)))


@pytest.mark.parametrize("ndim,order", [(2, 8), (3, 8), (2, 16), (3, 16)])
def test_host_cfl_matches_oracle(ndim, order):
    h = (10.0, 12.5, 7.5)
    a = fwi.fwi_cfl_number(ndim, order, h, 4500.0, 6e-4)
    b = oracle.cfl_number(ndim, order // 2, h, 4500.0, 6e-4)
    assert abs(a - b) <= 1e-6 * b


def test_cfl_limits_of_the_configs():
    # Courant limits with equal spacing (closed form of the stencil symbol at pi)
    for ndim, order, lim in [(2, 8, 0.5546), (3, 8, 0.4529), (2, 16, 0.5189), (3, 16, 0.4237)]:
        n = fwi.fwi_cfl_number(ndim, order, (1.0, 1.0, 1.0), 1.0, 1.0)
        assert abs(1.0 / n - lim) < 1e-4


# ------------------------------------------------------------------ checkpoint schedule

@lru_cache(maxsize=None)
def dp_min_steps(l, c):
    """Brute-force minimum forward steps to reverse l units with c free slots, S_first
    available (the recursion the schedule follows, minimised over every split)."""
    if l <= 1:
        return 0
    if c == 0:
        return l * (l - 1) // 2
    return min(t + dp_min_steps(l - t, c - 1) + dp_min_steps(t, c) for t in range(1, l))


def simulate(actions, nsteps, nslots):
    """Replays a schedule on symbolic states; returns (order of adjoint m, forward count)."""
    cur = 0
    slots = {}
    done = []
    fwd = 0
    for kind, arg in actions:
        if kind == 1:
            assert arg > 0
            cur += arg
            fwd += arg
            assert cur <= nsteps
        elif kind == 2:
            assert 0 <= arg < nslots
            slots[arg] = cur
        elif kind == 3:
            if arg == -1:
                cur = 0
            else:
                assert arg in slots, "restore of an empty slot"
                cur = slots[arg]
        elif kind == 4:
            assert cur == arg, f"adjoint {arg} with state {cur}"
            done.append(arg)
        else:
            raise AssertionError(kind)
    return done, fwd


@pytest.mark.parametrize("nsteps", [1, 2, 3, 7, 20, 55])
@pytest.mark.parametrize("nslots", [0, 1, 2, 3, 5, 60])
def test_revolve_schedule_is_valid_and_optimal(nsteps, nslots):
    acts, nf = fwi.fwi_revolve_schedule(nsteps, nslots)
    done, fwd = simulate(acts.tolist(), nsteps, nslots)
    assert done == list(range(nsteps, 0, -1))
    assert fwd == nf
    assert nf == dp_min_steps(nsteps + 1, min(nslots, nsteps + 1))


@pytest.mark.parametrize("nsteps,nslots", [(2000, 20), (4000, 40), (4000, 100), (3000, 7)])
def test_revolve_schedule_large(nsteps, nslots):
    from math import comb
    acts, nf = fwi.fwi_revolve_schedule(nsteps, nslots)
    done, fwd = simulate(acts.tolist(), nsteps, nslots)
    assert done == list(range(nsteps, 0, -1)) and fwd == nf
    # Griewank-Walther closed form T(l, c) = r l - binom(c + r + 1, c + 2)
    l, c = nsteps + 1, nslots
    r = 1
    while comb(c + 1 + r, c + 1) < l:
        r += 1
    assert nf == r * l - comb(c + 2 + r - 1, c + 2)


def _pair_slots(acts):
    """Slots that ever receive a pair, from the schedule alone: a restore followed by an
    adjoint step needs u^m only; a store needs the pair when a restore of another kind
    reads its slot before the slot's next store."""
    acts = [tuple(a) for a in acts]
    pairs = set()
    for i, (kind, arg) in enumerate(acts):
        if kind != 2:
            continue
        for k in range(i + 1, len(acts)):
            kk, aa = acts[k]
            if kk == 2 and aa == arg:
                break
            if kk == 3 and aa == arg and not (k + 1 < len(acts) and acts[k + 1][0] == 4):
                pairs.add(arg)
                break
    return pairs


@pytest.mark.parametrize("nsteps,halves", [(60, 200), (60, 59), (60, 40), (60, 8), (60, 1),
                                           (300, 45), (4000, 613), (3000, 2999)])
def test_checkpoint_plan_is_the_largest_layout_that_fits(nsteps, halves):
    slots, npair, nf = fwi.fwi_checkpoint_plan(nsteps, halves)
    acts, nf_ref = fwi.fwi_revolve_schedule(nsteps, slots)
    assert nf == nf_ref
    pairs = _pair_slots(acts.tolist())
    assert npair == len(pairs)
    assert slots + npair <= halves and slots <= nsteps
    if slots < nsteps:   # one more slot would not fit
        acts1, _ = fwi.fwi_revolve_schedule(nsteps, slots + 1)
        assert slots + 1 + len(_pair_slots(acts1.tolist())) > halves
    if halves >= nsteps - 1:   # u^n of every step fits: no recomputation, no pairs
        assert nf == nsteps and npair == 0


def test_checkpoint_plan_forward_steps_fall_with_budget():
    prev = None
    for halves in (0, 10, 50, 200, 613, 1200, 3999):
        nf = fwi.fwi_checkpoint_plan(4000, halves)[2]
        assert prev is None or nf <= prev
        prev = nf
    assert prev == 4000


@pytest.mark.parametrize("nsteps,pairs", [(500, 64), (3000, 64), (4000, 306), (4000, 20), (90, 8)])
def test_checkpoint_plan_never_worse_than_pair_slots(nsteps, pairs):
    """A budget of `pairs` pair-sized slots (2 * pairs units): sizing slots by what they
    hold gives at least as many slots and no more forward steps than pair slots alone."""
    slots, npair, nf = fwi.fwi_checkpoint_plan(nsteps, 2 * pairs)
    _, nf_pairs = fwi.fwi_revolve_schedule(nsteps, min(pairs, nsteps))
    assert slots >= min(pairs, nsteps) and nf <= nf_pairs


def test_host_functions_reject_bad_arguments():
    """Host-only entry points return FWI_ERR_ARG with a message for arguments outside their
    domain, and never touch the device."""
    with pytest.raises(fwi.FwiError) as e:
        fwi.fwi_revolve_schedule(0, 5)
    assert e.value.code == fwi.FWI_ERR_ARG and "nsteps" in fwi.fwi_last_error()
    with pytest.raises(fwi.FwiError) as e:
        fwi.fwi_checkpoint_plan(0, 10)
    assert e.value.code == fwi.FWI_ERR_ARG
    with pytest.raises(fwi.FwiError) as e:
        fwi.fwi_checkpoint_plan(10, -1)
    assert e.value.code == fwi.FWI_ERR_ARG
    for order in (0, 7, 40):
        with pytest.raises(fwi.FwiError) as e:
            fwi.fwi_fd_coeffs(order)
        assert e.value.code == fwi.FWI_ERR_ARG
    assert fwi.fwi_cfl_number(4, 8, (10.0, 10.0, 10.0), 3000.0, 1e-3) < 0      # bad ndim
    assert fwi.fwi_cfl_number(3, 9, (10.0, 10.0, 10.0), 3000.0, 1e-3) < 0      # odd order
