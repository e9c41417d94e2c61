"""Temporal blocking of the 2-D forward step (fwi_opts.temporal_blocking).  Mode 1: a batch
of shots wide enough to fill the GPU advances two time steps per pass; its traces and final
state equal the single-step path (each shot on its own, too few shots for the two-step
pass) bit for bit, including an odd step count (the last step single), and match the FP64
oracle.  Mode 2: a one-shot request small enough for one cluster of CTAs advances up to 64
steps per launch with its states in shared memory; the same bars."""
import numpy as np
import pytest

import oracle
from paper_1912_08063_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _case(order, nshots, nt, seed):
    rng = np.random.default_rng(seed)
    nz, nx = 96, 200
    h = 10.0
    v = synth.smooth_random(rng, (nz, nx), h, ell=150.0)
    dt = 0.4 * h / 4500.0
    src = np.stack([np.full(nshots, 6), np.zeros(nshots, int),
                    rng.integers(0, nx, nshots)], 1).astype(np.int32)
    rec = np.stack([np.full(40, 3), np.zeros(40, int), np.linspace(0, nx - 1, 40).astype(int)],
                   1).astype(np.int32)
    wav = np.stack([synth.ricker(25.0, dt, nt) * (1 + 0.01 * s) for s in range(nshots)])
    return v, h, dt, src, rec, wav.astype(np.float32)


@pytest.mark.parametrize("order,nshots,nt", [(8, 48, 61), (16, 80, 40)])
def test_two_step_pass_equals_single_steps(order, nshots, nt):
    from paper_1912_08063_gb300 import fwi
    v, h, dt, src, rec, wav = _case(order, nshots, nt, seed=order)
    m = fwi.FwiModel(torch.from_numpy(v).cuda(), h, dt, nt, order=order, sponge_vref=4600.0,
                     temporal_blocking=True)
    tr, fin = m.forward(fwi.Acquisition(src, rec), torch.from_numpy(wav).cuda(), final_state=True)
    tr, fin = tr.cpu().numpy(), fin.cpu().numpy()
    for s in (0, nshots // 2, nshots - 1):
        t1, f1 = m.forward(fwi.Acquisition(src[s:s + 1], rec), torch.from_numpy(wav[s:s + 1]).cuda(),
                           final_state=True)
        assert np.array_equal(tr[s], t1.cpu().numpy()[0])
        assert np.array_equal(fin[s], f1.cpu().numpy()[0])


def test_two_step_pass_matches_oracle():
    from paper_1912_08063_gb300 import fwi
    nshots, nt = 48, 50
    v, h, dt, src, rec, wav = _case(8, nshots, nt, seed=3)
    m = fwi.FwiModel(torch.from_numpy(v).cuda(), h, dt, nt, order=8, sponge_vref=4600.0,
                     temporal_blocking=True)
    tr = m.forward(fwi.Acquisition(src, rec), torch.from_numpy(wav).cuda()).cpu().numpy()
    pick = [0, 17, 47]
    P = oracle.Problem(v, (h, h), dt, nt, order=8, nb=20, vref=4600.0, src=src[pick], rec=rec,
                       wavelet=wav[pick].astype(np.float64))
    ref = P.forward()
    e = np.linalg.norm(tr[pick] - ref) / np.linalg.norm(ref)
    print(f"two-step pass traces vs oracle: rel-L2 {e:.2e}")
    assert e <= 1e-4


@pytest.mark.parametrize("shape,order", [((60, 90), 8), ((131, 77), 16), ((300, 280), 8)])
def test_onchip_blocking_equals_single_steps(shape, order):
    """temporal_blocking = 2: a one-shot 2-D forward with receivers on one row runs up to
    64 steps per launch in one cluster of CTAs with both states in shared memory; traces
    and the final state equal single steps bit for bit, and the traces match the
    oracle."""
    from paper_1912_08063_gb300 import fwi
    import oracle
    rng = np.random.default_rng(41)
    nz, nx = shape
    v = synth.smooth_random(rng, shape, 10.0, ell=80.0)
    h, nt = 10.0, 150
    dt = 0.5 / fwi.fwi_cfl_number(2, order, (h, h, h), float(v.max()), 1.0)
    src = np.array([[3, 0, nx // 2]], dtype=np.int32)
    rec = np.array([[2, 0, x] for x in range(nx)], dtype=np.int32)
    wav = synth.ricker(25.0, dt, nt)[None].astype(np.float32)
    acq = fwi.Acquisition(src, rec)
    outs = []
    for tb in (0, 2):
        m = fwi.FwiModel(torch.from_numpy(v).cuda(), h, dt, nt, order=order, nb=20,
                         temporal_blocking=tb)
        tr, fin = m.forward(acq, torch.from_numpy(wav).cuda(), final_state=True)
        outs.append((tr.cpu().numpy(), fin.cpu().numpy()))
        m.close()
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    ref = oracle.Problem(v, h, dt, nt, order=order, nb=20, src=src, rec=rec,
                         wavelet=wav).forward()
    e = np.linalg.norm(outs[1][0] - ref) / np.linalg.norm(ref)
    print(f"on-chip blocking {shape} order {order}: traces rel-L2 {e:.2e}")
    assert e <= 1e-4
