"""FWI outer loop: the host logic on an analytic problem (CPU) and a few iterations on
the GPU that must lower the misfit and bring the model closer to the true one."""
import numpy as np
import pytest

from paper_1912_08063_gb300 import invert, synth


def test_descend_on_a_quadratic():
    """phi(v) = sum w (v - v*)^2 with a box: the loop decreases phi monotonically and
    converges to the box-clipped minimiser."""
    rng = np.random.default_rng(0)
    vstar = rng.uniform(1400.0, 4600.0, 50)
    wts = rng.uniform(0.5, 2.0, 50)
    f = lambda v: (float(np.sum(wts * (v - vstar) ** 2)), 2 * wts * (v - vstar))
    v, hist = invert.descend(np.full(50, 3000.0), f, iters=200, max_dv=200.0)
    assert all(b <= a for a, b in zip(hist, hist[1:]))
    assert np.allclose(v, np.clip(vstar, 1500.0, 4500.0), atol=1.0)


@pytest.mark.gpu
def test_fwi_iterations_reduce_misfit_and_model_error():
    torch = pytest.importorskip("torch")
    from paper_1912_08063_gb300 import fwi
    rng = np.random.default_rng(3)
    nz, nx = 60, 100
    vtrue = np.full((nz, nx), 2000.0, dtype=np.float32)
    vtrue[30:, :] = 2600.0
    vtrue[20:26, 40:60] = 2300.0                      # a small anomaly to recover
    v0 = np.full((nz, nx), 2000.0, dtype=np.float32)
    v0[30:, :] = 2600.0
    h, dt, nt = 10.0, 1e-3, 400
    src = np.array([[2, 0, x] for x in (10, 50, 90)], dtype=np.int32)
    rec = np.stack([np.full(nx, 2), np.zeros(nx), np.arange(nx)], 1).astype(np.int32)
    wav = torch.from_numpy(np.broadcast_to(synth.ricker(15.0, dt, nt), (3, nt)).copy()).cuda()
    acq = fwi.Acquisition(src, rec)
    obs = fwi.FwiModel(torch.from_numpy(vtrue).cuda(), h, dt, nt, sponge_vref=4500.0)
    dobs = obs.forward(acq, wav)
    m = fwi.FwiModel(torch.from_numpy(v0).cuda(), h, dt, nt, sponge_vref=4500.0)
    f = invert.gpu_evaluator(m, acq, wav, dobs)
    v, hist = invert.descend(torch.from_numpy(v0).cuda(), f, iters=4, max_dv=60.0)
    err0 = np.linalg.norm(v0 - vtrue)
    err1 = np.linalg.norm(v.cpu().numpy() - vtrue)
    print(f"FWI misfit {hist}, model error {err0:.1f} -> {err1:.1f}")
    assert len(hist) >= 3 and hist[-1] < 0.7 * hist[0]
    assert err1 < err0
