"""Parity at the full size of the benchmark workload (the 512^3 salt model, 16th order,
20-cell sponge, 256 x 256 receivers) in the launch configuration bench.py times.

The oracle cannot run a 552^3 grid for long, but it does not need to: after K steps the
field is non-zero only within K*M cells (L1 distance) of the source, because each step
widens the support by the stencil radius M along one axis.  A crop of the model that
shares the real top face (so the top sponge is the same) and reaches further than that
radius on every other side gives, in exact arithmetic, the same wavefield, traces and
(for the reverse sweep, whose support is within 2*K*M cells) the same gradient.  So the
GPU's full-size results are compared with the oracle's on the crop, element by element.
"""
import numpy as np
import pytest

import oracle
from paper_1912_08063_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K = 6          # time steps
VREF = 4500.0  # the sponge strength the bench uses


@pytest.fixture(scope="module")
def salt512():
    return synth.salt_3d(512)


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _crop_problem(w, half, depth, wav, rec_full):
    sz, sy, sx = (int(x) for x in w.src[0])
    y0, x0 = sy - half, sx - half
    v = np.ascontiguousarray(w.v[:depth, y0:y0 + 2 * half + 1, x0:x0 + 2 * half + 1], np.float64)
    inside = ((rec_full[:, 0] < depth) & (rec_full[:, 1] >= y0) & (rec_full[:, 1] <= y0 + 2 * half)
              & (rec_full[:, 2] >= x0) & (rec_full[:, 2] <= x0 + 2 * half))
    rec = rec_full[inside] - np.array([0, y0, x0])
    p = oracle.Problem(v, w.h, w.dt, K, order=w.order, nb=w.nb, vref=VREF,
                       src=[[sz, sy - y0, sx - x0]], rec=rec, wavelet=wav)
    return p, inside, (y0, x0)


def test_forward_fullsize_512(salt512):
    from paper_1912_08063_gb300 import fwi
    w = salt512
    rng = np.random.default_rng(512)
    wav = rng.standard_normal((1, K)).astype(np.float32)
    m = fwi.FwiModel(torch.from_numpy(w.v).cuda(), w.h, w.dt, K, order=w.order, nb=w.nb,
                     sponge_vref=VREF)
    acq = fwi.Acquisition(w.src, w.rec)
    tr, fin = m.forward(acq, torch.from_numpy(wav).cuda(), final_state=True)
    M = w.order // 2
    half, depth = K * M + 4, int(w.src[0, 0]) + K * M + 4
    p, inside, (y0, x0) = _crop_problem(w, half, depth, wav, w.rec)
    rtr, rfin = p.forward(final=True)
    nb = w.nb
    # the crop's computed grid sits at computed rows [0, depth + nb) of the full grid and
    # computed columns [y0, y0 + 2 half + 1 + 2 nb) (the crop is padded by nb too)
    g = fin[0, :, : depth + nb, y0: y0 + 2 * half + 1 + 2 * nb,
            x0: x0 + 2 * half + 1 + 2 * nb].cpu().numpy()
    # compare only where the full-grid crop is the oracle's physical region plus the real
    # top sponge (the oracle's own lateral/bottom sponge cells carry no field)
    o = rfin[0]
    sl = (slice(None), slice(0, depth + nb), slice(nb, nb + 2 * half + 1), slice(nb, nb + 2 * half + 1))
    e_fin = rel(g[sl], o[sl])
    e_tr = rel(tr.cpu().numpy()[0][:, inside], rtr[0])
    outside = np.abs(tr.cpu().numpy()[0][:, ~inside]).max()
    print(f"512^3 forward, {K} steps: final field rel-L2 {e_fin:.2e}, traces {e_tr:.2e}, "
          f"max |trace| outside the support {outside:.1e}")
    assert e_fin <= 1e-4 and e_tr <= 1e-4
    assert outside == 0.0
    m.close()


@pytest.mark.parametrize("snap,tol", [("fp32", 1e-3), ("fp16", 1e-2)])
def test_gradient_fullsize_512(salt512, snap, tol):
    from paper_1912_08063_gb300 import fwi
    w = salt512
    rng = np.random.default_rng(513)
    wav = rng.standard_normal((1, K)).astype(np.float32)
    m = fwi.FwiModel(torch.from_numpy(w.v).cuda(), w.h, w.dt, K, order=w.order, nb=w.nb,
                     sponge_vref=VREF, snap_dtype=snap, snap_budget_bytes=2 * 673 * 2 ** 20)
    acq = fwi.Acquisition(w.src, w.rec)
    dobs = np.zeros((1, K, w.nrec), dtype=np.float32)   # residual = data
    phi, g = m.gradient(acq, torch.from_numpy(wav).cuda(), torch.from_numpy(dobs).cuda())
    info = m.info()
    M = w.order // 2
    half, depth = 2 * K * M + 4, int(w.src[0, 0]) + 2 * K * M + 4
    p, inside, (y0, x0) = _crop_problem(w, half, depth, wav, w.rec)
    rphi, rg = p.gradient(np.zeros((1, K, int(inside.sum()))))
    gg = g.cpu().numpy()
    crop = gg[:depth, y0:y0 + 2 * half + 1, x0:x0 + 2 * half + 1]
    e = rel(crop, rg)
    mask = np.ones(gg.shape, dtype=bool)
    mask[:depth, y0:y0 + 2 * half + 1, x0:x0 + 2 * half + 1] = False
    rest = float(np.abs(gg[mask]).max())
    print(f"512^3 gradient ({snap} checkpoints, {info['snap_slots']} slots, "
          f"{info['last_forward_steps']} forward steps): rel-L2 {e:.2e}, misfit rel "
          f"{abs(phi.item() - rphi) / rphi:.2e}, |g| outside the support {rest:.1e}")
    assert e <= tol
    assert abs(phi.item() - rphi) <= tol * rphi
    assert rest == 0.0
    m.close()
