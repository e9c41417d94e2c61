"""Failure paths reached on purpose without a GPU fault: a bounded device wait that runs
out (FWI_ERR_TIMEOUT, latched per model) and a memory budget too small for a request
(FWI_ERR_OOM before anything is launched for it)."""
import math

import numpy as np
import pytest

from paper_1912_08063_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _small_model(fwi, rng):
    w = synth.random_small(rng, 3, (20, 18, 22), nt=30, nb=4, nrec=5)
    m = fwi.FwiModel(torch.from_numpy(w.v).cuda(), w.h, w.dt, w.nt, order=8, nb=w.nb)
    return w, m


def test_bounded_wait_runs_out_and_latches_timeout():
    from paper_1912_08063_gb300 import fwi
    rng = np.random.default_rng(21)
    w, m = _small_model(fwi, rng)
    acq = fwi.Acquisition(w.src, w.rec)
    wav = torch.from_numpy(w.wavelets()).cuda()
    before = m.forward(acq, wav).cpu().numpy()
    fwi.fwi_sync_status(m.handle)                   # clean so far
    fwi.fwi_selftest_wait(m.handle, 10_000)         # an mbarrier whose bytes never land
    with pytest.raises(fwi.FwiError) as e:
        fwi.fwi_sync_status(m.handle)
    assert e.value.code == fwi.FWI_ERR_TIMEOUT
    with pytest.raises(fwi.FwiError) as e:          # latched: later calls report it too
        m.forward(acq, wav)
    assert e.value.code == fwi.FWI_ERR_TIMEOUT
    m.close()
    # the context is intact: a fresh model computes the same traces
    m2 = fwi.FwiModel(torch.from_numpy(w.v).cuda(), w.h, w.dt, w.nt, order=8, nb=w.nb)
    after = m2.forward(acq, wav).cpu().numpy()
    fwi.fwi_sync_status(m2.handle)
    m2.close()
    assert np.array_equal(before, after)


def test_selftest_rejects_poll_limits_out_of_range():
    from paper_1912_08063_gb300 import fwi
    w, m = _small_model(fwi, np.random.default_rng(22))
    for polls in (0, -5, (1 << 22) + 1):
        with pytest.raises(fwi.FwiError) as e:
            fwi.fwi_selftest_wait(m.handle, polls)
        assert e.value.code == fwi.FWI_ERR_ARG
    fwi.fwi_sync_status(m.handle)                   # nothing was launched
    m.close()


def test_serving_budget_smaller_than_a_request_is_oom():
    from paper_1912_08063_gb300 import fwi

    def dt_for(ndim, h):
        lim = 1.0 / fwi.fwi_cfl_number(ndim, 8, (h, h, h), 4500.0, 1.0)
        return math.floor(0.8 * lim * 1e4) / 1e4

    reqs = synth.serving_requests(4, dt_for, seed=3, size2d=(40, 60), size3d=(20, 24),
                                  nt_range=(20, 40))
    for r in reqs:
        r["arrival"] = 0.0
        if r["kind"] == "gradient":
            r["d_obs"] = np.zeros((r["nt"], len(r["rec"])), dtype=np.float32)
    one_field = 4 * 60 * 60    # smaller than any request's wavefield
    res, out = fwi.fwi_serve(reqs, budget_bytes=one_field, max_active=4, snap_slots=2)
    for x, o in zip(res, out):
        assert x["status"] == fwi.FWI_ERR_OOM, x
        assert x["device_bytes"] == 0 and x["t_admit"] == 0.0   # never admitted
        assert not np.any(o)
