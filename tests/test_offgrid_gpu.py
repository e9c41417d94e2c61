"""GPU parity for off-grid sources and receivers (Kaiser-windowed sinc points): traces,
gradients and the wavelet-space adjoint against the FP64 oracle on the same positions.
Bars as for on-grid points: traces rel-L2 <= 1e-4, FP32-checkpoint gradients <= 1e-3,
BF16 checkpoints <= 1e-2."""
import numpy as np
import pytest

import oracle
from paper_1912_08063_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _case(ndim, shape, order, nshots=2, nrec=6, nt=70, seed=0, nb=20, margin=0.0):
    """Random smooth model, fractional source/receiver positions anywhere in the physical
    grid (within `margin` of the faces)."""
    rng = np.random.default_rng(seed + 10 * ndim + order)
    h = 10.0
    v = synth.smooth_random(rng, shape, h, ell=80.0)
    dt = 0.4 * h / 4500.0

    def pos(n):
        p = np.stack([rng.uniform(margin, s - 1 - margin, n) for s in shape], axis=1)
        if ndim == 2:
            p = np.stack([p[:, 0], np.zeros(n), p[:, 1]], axis=1)
        return p

    src_pos = pos(nshots)
    rec_pos = pos(nshots * nrec).reshape(nshots, nrec, 3)
    wav = np.stack([synth.ricker(30.0, dt, nt) * (1.0 + 0.3 * s) for s in range(nshots)])
    return dict(v=v, h=h, dt=dt, nt=nt, order=order, nb=nb, src_pos=src_pos,
                rec_pos=rec_pos, wav=wav.astype(np.float32), rng=rng)


def _gpu(c, snap="fp32", v=None):
    from paper_1912_08063_gb300 import fwi
    v = c["v"] if v is None else v
    m = fwi.FwiModel(torch.from_numpy(np.ascontiguousarray(v, dtype=np.float32)).cuda(),
                     c["h"], c["dt"], c["nt"], order=c["order"], nb=c["nb"],
                     sponge_vref=4600.0, snap_dtype=snap)
    acq = fwi.Acquisition(src_pos=c["src_pos"], rec_pos=c["rec_pos"])
    return m, acq


def _oracle(c, v=None):
    v = c["v"] if v is None else v
    return oracle.Problem(v, c["h"], c["dt"], c["nt"], order=c["order"], nb=c["nb"],
                          vref=4600.0, src_pos=c["src_pos"], rec_pos=c["rec_pos"],
                          wavelet=c["wav"].astype(np.float64))


@pytest.mark.parametrize("ndim,shape,order", [
    (2, (37, 45), 8), (2, (30, 34), 16), (3, (15, 17, 19), 8), (3, (13, 14, 16), 16)])
def test_offgrid_forward_traces(ndim, shape, order):
    c = _case(ndim, shape, order)
    m, acq = _gpu(c)
    tr = m.forward(acq, torch.from_numpy(c["wav"]).cuda()).cpu().numpy()
    ref = _oracle(c).forward()
    e = rel(tr, ref)
    print(f"off-grid traces {ndim}d o{order}: rel-L2 {e:.2e}")
    assert e <= 1e-4


@pytest.mark.parametrize("ndim,shape,order,snap,tol", [
    (2, (31, 39), 8, "fp32", 1e-3), (3, (13, 15, 17), 16, "fp32", 1e-3),
    (2, (33, 41), 8, "bf16", 1e-2), (3, (14, 15, 16), 8, "fp16", 1e-2)])
def test_offgrid_gradient(ndim, shape, order, snap, tol):
    c = _case(ndim, shape, order, nt=60)
    vobs = c["v"] * (1.0 + 0.04 * synth.gaussian_random_field(c["rng"], c["v"].shape, c["h"], 40.0, 1.0))
    dobs = _oracle(c, v=vobs).forward().astype(np.float32)
    m, acq = _gpu(c, snap=snap)
    phi, g = m.gradient(acq, torch.from_numpy(c["wav"]).cuda(), torch.from_numpy(dobs).cuda())
    rphi, rg = _oracle(c).gradient(dobs.astype(np.float64))
    e = rel(g.cpu().numpy(), rg)
    print(f"off-grid gradient {ndim}d o{order} {snap}: rel-L2 {e:.2e}")
    assert e <= tol
    assert abs(phi.item() - rphi) <= 1e-3 * rphi


def test_offgrid_source_adjoint_matches_oracle():
    c = _case(2, (29, 35), 8, nt=50)
    m, acq = _gpu(c)
    y = c["rng"].standard_normal((2, c["nt"], 6)).astype(np.float32)
    x = m.source_adjoint(acq, torch.from_numpy(y).cuda()).cpu().numpy()
    ref = _oracle(c).source_adjoint(y.astype(np.float64))
    print(f"off-grid source adjoint: rel-L2 {rel(x, ref):.2e}")
    assert rel(x, ref) <= 1e-4


def test_integer_positions_match_nodes():
    """Positions on nodes give the node results (to FP32 rounding: the tap injection runs
    after the step instead of inside it)."""
    from paper_1912_08063_gb300 import fwi
    c = _case(3, (12, 13, 14), 8, nshots=1)
    src = np.rint(c["src_pos"]).astype(np.int32)
    rec = np.rint(c["rec_pos"]).astype(np.int32)
    m, _ = _gpu(c)
    wav = torch.from_numpy(c["wav"][:1]).cuda()
    t_nodes = m.forward(fwi.Acquisition(src, rec), wav).cpu().numpy()
    t_pos = m.forward(fwi.Acquisition(src_pos=src.astype(np.float64),
                                      rec_pos=rec.astype(np.float64)), wav).cpu().numpy()
    assert rel(t_pos, t_nodes) <= 1e-6


def test_offgrid_point_outside_is_rejected():
    from paper_1912_08063_gb300 import fwi
    c = _case(2, (20, 24), 8, nshots=1, nb=2)
    m, _ = _gpu(c)
    wav = torch.from_numpy(c["wav"][:1]).cuda()
    bad = fwi.Acquisition(src_pos=np.array([[0.5, 0.0, 10.0]]),
                          rec_pos=np.array([[[5.0, 0.0, 5.0]]]))   # taps cross the grid edge
    with pytest.raises(RuntimeError):
        m.forward(bad, wav)
