"""GPU parity: the CUDA path (called through the C ABI) against the FP64 oracle on the
same seeded inputs.  Bars: traces and final wavefields rel-L2 <= 1e-4; gradients
rel-L2 <= 1e-3 with FP32 checkpoints and <= 1e-2 with BF16/FP16 checkpoints; codec
bit-exact; misfit rel <= 1e-6."""
import numpy as np
import pytest

import oracle
from paper_1912_08063_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FWD = 1e-4
TOL_GRAD32 = 1e-3
TOL_GRAD16 = 1e-2


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def fwi():
    from paper_1912_08063_gb300 import fwi as f
    return f


def make_pair(w, vref=4600.0, snap="fp32", budget=0, nb=None, v=None, order=None):
    f = fwi()
    nb = w.nb if nb is None else nb
    v = w.v if v is None else v
    m = f.FwiModel(torch.from_numpy(np.ascontiguousarray(v)).cuda(), w.h, w.dt, w.nt,
                   order=w.order, nb=nb, sponge_vref=vref, snap_dtype=snap,
                   snap_budget_bytes=budget)
    p = oracle.Problem(v, w.h, w.dt, w.nt, order=w.order, nb=nb, vref=vref, src=w.src,
                       rec=w.rec, wavelet=w.wavelets())
    return m, p, f.Acquisition(w.src, w.rec)


def gpu_forward(m, acq, w, final=True):
    wav = torch.from_numpy(w.wavelets()).cuda()
    out = m.forward(acq, wav, final_state=final)
    if final:
        return out[0].cpu().numpy(), out[1].cpu().numpy()
    return out.cpu().numpy()


# ------------------------------------------------------------------ forward

def test_forward_two_layer_2d():
    """2-D two-layer model, 201 x 201, 8th order, dt 1 ms, 500 steps, 15 Hz Ricker."""
    w = synth.two_layer_2d()
    m, p, acq = make_pair(w)
    tr, fin = gpu_forward(m, acq, w)
    rtr, rfin = p.forward(final=True)
    e_tr, e_fin = rel(tr, rtr), rel(fin.reshape(rfin.shape), rfin)
    print(f"two_layer_2d: traces {e_tr:.2e} final {e_fin:.2e}")
    assert e_tr <= TOL_FWD and e_fin <= TOL_FWD


CASES = [
    # ndim, physical shape, order, nb — ragged sizes that span several tiles
    (2, (37, 45), 8, 6),
    (2, (19, 300), 16, 5),
    (2, (70, 131), 8, 0),
    (3, (23, 17, 41), 8, 4),
    (3, (15, 21, 29), 16, 3),
    (3, (9, 40, 33), 8, 0),
    (3, (6, 5, 7), 16, 0),        # grid smaller than the stencil radius
]


@pytest.mark.parametrize("ndim,shape,order,nb", CASES)
def test_forward_random_models(ndim, shape, order, nb):
    rng = np.random.default_rng(hash((ndim, shape, order)) & 0xffff)
    w = synth.random_small(rng, ndim, shape, nt=50, order=order, nb=nb, nrec=11)
    # receivers on the grid corners and on tile edges too
    extra = [[0, 0, 0], [shape[0] - 1, 0 if ndim == 2 else shape[1] - 1, shape[-1] - 1]]
    if shape[-1] > 32:
        extra.append([shape[0] // 2, 0 if ndim == 2 else shape[1] // 2, 31 - nb if nb < 31 else 0])
    w.rec = np.concatenate([w.rec, np.array(extra, dtype=np.int32)], 0)
    m, p, acq = make_pair(w)
    tr, fin = gpu_forward(m, acq, w)
    rtr, rfin = p.forward(final=True)
    e_tr, e_fin = rel(tr, rtr), rel(fin.reshape(rfin.shape), rfin)
    print(f"forward {ndim}d {shape} o{order} nb{nb}: traces {e_tr:.2e} final {e_fin:.2e}")
    assert e_tr <= TOL_FWD and e_fin <= TOL_FWD, (e_tr, e_fin)


def test_forward_batched_shots_2d():
    w = synth.faulted_2d(nz=60, nx=160, nt=120, nshots=5)
    w.nb = 8
    m, p, acq = make_pair(w)
    tr, fin = gpu_forward(m, acq, w)
    rtr, rfin = p.forward(final=True)
    e_tr, e_fin = rel(tr, rtr), rel(fin.reshape(rfin.shape), rfin)
    print(f"forward 2d 5 batched shots: traces {e_tr:.2e} final {e_fin:.2e}")
    assert e_tr <= TOL_FWD and e_fin <= TOL_FWD


def test_forward_single_step_and_host_buffers():
    """nt = 1 (one update from rest: only the source node is non-zero) through host
    (numpy) buffers."""
    f = fwi()
    rng = np.random.default_rng(4)
    w = synth.random_small(rng, 3, (11, 12, 13), nt=1, nb=2, nrec=4)
    m = f.FwiModel(w.v, w.h, w.dt, w.nt, order=8, nb=w.nb, sponge_vref=4600.0)
    acq = f.Acquisition(w.src, w.rec)
    tr = np.zeros((1, 1, w.nrec), dtype=np.float32)
    f.fwi_forward(m.handle, acq.c, w.wavelets(), tr)
    p = oracle.Problem(w.v, w.h, w.dt, 1, order=8, nb=w.nb, vref=4600.0, src=w.src,
                       rec=w.rec, wavelet=w.wavelets())
    assert rel(tr, p.forward()) <= TOL_FWD or np.abs(p.forward()).max() == 0


# ------------------------------------------------------------------ misfit and codec

def test_misfit_matches_oracle():
    f = fwi()
    rng = np.random.default_rng(8)
    for n in (1, 1000, 123457, 3_000_001):
        a = rng.standard_normal(n).astype(np.float32)
        b = (a + 1e-3 * rng.standard_normal(n)).astype(np.float32)
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        f.fwi_misfit(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), n, out)
        # the oracle takes the FP32 residual the kernel forms, then sums in FP64
        r = (a - b).astype(np.float64)
        ref = oracle.misfit(r, np.zeros_like(r))
        # same terms, different FP64 summation order: |error| <= n eps sum|terms|
        print(f"misfit n={n}: rel {abs(out.item() - ref) / ref:.2e}")
        assert abs(out.item() - ref) <= n * 2.0 ** -52 * ref


@pytest.mark.parametrize("dtype", ["bf16", "fp16"])
def test_codec_bit_exact(dtype):
    f = fwi()
    rng = np.random.default_rng(9)
    n = 100_003
    a = (rng.standard_normal(n) * 10.0 ** rng.uniform(-9, -3, n)).astype(np.float32)
    b = (rng.standard_normal(n) * 1e-6).astype(np.float32)
    a[:5] = [0.0, -0.0, 1e-30, -2.0 ** -20, 3.3e-3]
    code = torch.zeros(2 * n, dtype=torch.int16, device="cuda")
    sc = torch.zeros(2, dtype=torch.float32, device="cuda")
    ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    dt_id = {"bf16": 1, "fp16": 2}[dtype]
    f.fwi_snapshot_encode(ta, tb, n, dt_id, code, sc)
    rcode, rs = oracle.snap_encode(a, b, dtype)
    assert np.array_equal(sc.cpu().numpy(), rs)
    assert np.array_equal(code.cpu().numpy().view(np.uint16).reshape(2, n), rcode)
    da, db = torch.empty_like(ta), torch.empty_like(tb)
    f.fwi_snapshot_decode(code, sc, n, dt_id, da, db)
    ra, rb = oracle.snap_decode(rcode, rs, dtype)
    assert np.array_equal(da.cpu().numpy(), ra) and np.array_equal(db.cpu().numpy(), rb)


# ------------------------------------------------------------------ adjoint and gradient

@pytest.mark.parametrize("ndim,shape,order", [(2, (30, 41), 8), (3, (13, 14, 19), 16)])
def test_source_dot_product_gpu(ndim, shape, order):
    """<F x, y> = <x, F* y> for the GPU forward and GPU source adjoint (FP32 arithmetic,
    FP64 dots)."""
    rng = np.random.default_rng(12)
    w = synth.random_small(rng, ndim, shape, nt=60, order=order, nb=5, nrec=9)
    f = fwi()
    m, p, acq = make_pair(w)
    x = rng.standard_normal((1, w.nt)).astype(np.float32)
    y = rng.standard_normal((1, w.nt, w.nrec)).astype(np.float32)
    Fx = m.forward(acq, torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    Fty = m.source_adjoint(acq, torch.from_numpy(y).cuda()).cpu().numpy().astype(np.float64)
    lhs, rhs = np.sum(Fx * y), np.sum(x * Fty)
    ref = p.source_adjoint(y.astype(np.float64))
    print(f"dot product {ndim}d o{order}: rel {abs(lhs - rhs) / max(abs(lhs), abs(rhs)):.2e}, "
          f"source adjoint vs oracle {rel(Fty, ref):.2e}")
    assert abs(lhs - rhs) <= 1e-5 * max(abs(lhs), abs(rhs)), (lhs, rhs)
    # and the GPU source adjoint against the oracle's
    assert rel(Fty, ref) <= TOL_FWD


def _grad_case(ndim, shape, order, nt=70, nb=5, seed=13, nshots=1, f0=20.0):
    rng = np.random.default_rng(seed)
    w = synth.random_small(rng, ndim, shape, nt=nt, order=order, nb=nb, nrec=12, f0=f0)
    if nshots > 1:
        src = np.repeat(w.src, nshots, 0)
        src[:, -1] = rng.integers(0, shape[-1], nshots)
        w.src = src
    # observed data from a model 10 % slower with 5 % random variations: the residual is
    # a sizeable fraction of the data, as in an FWI iteration (a residual of ~1 % of the
    # data would turn FP32 rounding of the traces into ~1e-4 misfit differences)
    vobs = w.v * (0.9 + 0.05 * synth.gaussian_random_field(rng, w.v.shape, w.h, 40.0, 1.0))
    p_obs = oracle.Problem(vobs, w.h, w.dt, w.nt, order=order, nb=nb, vref=4600.0,
                           src=w.src, rec=w.rec, wavelet=w.wavelets())
    dobs = p_obs.forward().astype(np.float32)
    return w, dobs


@pytest.mark.parametrize("ndim,shape,order,nshots", [
    (2, (33, 47), 8, 1), (2, (29, 38), 16, 3), (3, (14, 17, 21), 8, 1), (3, (12, 13, 15), 16, 2)])
def test_gradient_fp32_checkpoints(ndim, shape, order, nshots):
    w, dobs = _grad_case(ndim, shape, order, nshots=nshots)
    m, p, acq = make_pair(w, snap="fp32")
    phi, g = m.gradient(acq, torch.from_numpy(w.wavelets()).cuda(), torch.from_numpy(dobs).cuda())
    rphi, rg = p.gradient(dobs.astype(np.float64))
    e = rel(g.cpu().numpy(), rg)
    rr = np.sqrt(rphi) / np.linalg.norm(dobs)
    print(f"grad fp32 {ndim}d o{order}: rel-L2 {e:.2e}, misfit rel "
          f"{abs(phi.item() - rphi) / rphi:.2e}, |r|/|d_obs| {rr:.2f}")
    assert e <= TOL_GRAD32
    assert abs(phi.item() - rphi) <= TOL_GRAD32 * rphi


def test_gradient_independent_of_checkpoint_budget_fp32():
    """With FP32 checkpoints restores are exact, so every budget (no checkpoint, a few,
    one per step) gives the same gradient bit for bit."""
    w, dobs = _grad_case(2, (25, 31), 8, nt=40)
    grads = []
    for budget in (0, 1, 3 * 2 * 4 * (41 * 44 + 64), 10 ** 9):
        m, p, acq = make_pair(w, snap="fp32", budget=budget if budget else 1)
        _, g = m.gradient(acq, torch.from_numpy(w.wavelets()).cuda(), torch.from_numpy(dobs).cuda())
        grads.append(g.cpu().numpy())
        info = m.info()
        assert info["last_adjoint_steps"] == w.nt
    for g in grads[1:]:
        assert np.array_equal(g, grads[0])


def _config_case(w, nslots, snap):
    """GPU and oracle gradients of workload w with nslots 16-bit checkpoints; d_obs from
    the oracle on w.v_obs."""
    vref = 4600.0
    p_obs = oracle.Problem(w.v_obs, w.h, w.dt, w.nt, order=w.order, nb=w.nb, vref=vref,
                           src=w.src, rec=w.rec, wavelet=w.wavelets())
    dobs = p_obs.forward().astype(np.float32)
    probe, _, _ = make_pair(w, snap=snap, budget=1, vref=vref)
    pitch, comp = probe.info()["pitch_x"], probe.info()["computed"]
    field = -(-comp[0] * comp[1] * pitch // 64) * 64
    m, p, acq = make_pair(w, snap=snap, budget=nslots * 2 * 2 * field, vref=vref)
    phi, g = m.gradient(acq, torch.from_numpy(w.wavelets()).cuda(), torch.from_numpy(dobs).cuda())
    info = m.info()
    rphi, rg = p.gradient(dobs.astype(np.float64))
    return rel(g.cpu().numpy(), rg), info, abs(phi.item() - rphi) / rphi


def test_gradient_layered_64_instance_bf16():
    """64^3 instance of the 256^3 layered model (h 10 m, dt 0.8 ms, 8th order, 15 Hz,
    receivers every 2nd cell on row 5), 300 steps, a budget of 20 BF16 pair checkpoints
    (more slots than 20 once those that only ever hold u^n take one field)."""
    w = synth.layered_3d(64, nt=300)
    e, info, em = _config_case(w, 20, "bf16")
    print(f"layered 64^3 bf16: grad rel-L2 {e:.2e}, misfit rel {em:.2e}, "
          f"slots {info['snap_slots']}, forward steps {info['last_forward_steps']}")
    slots, _, nf = fwi().fwi_checkpoint_plan(w.nt, 40)
    assert info["snap_slots"] == slots >= 20 and info["last_forward_steps"] == nf > w.nt
    assert e <= TOL_GRAD16


def test_gradient_salt_96_twin_fp16():
    """96^3 twin of the 512^3 salt model (h and dt scaled by 512/96, 16th order, FP16
    checkpoints), the first 250 steps, 12 checkpoints."""
    w = synth.salt_3d(96)
    w.nt = 250
    e, info, em = _config_case(w, 12, "fp16")
    print(f"salt 96^3 fp16: grad rel-L2 {e:.2e}, misfit rel {em:.2e}, "
          f"slots {info['snap_slots']}, forward steps {info['last_forward_steps']}")
    assert e <= TOL_GRAD16


def test_autograd_matches_finite_difference():
    """WaveFwi.apply/backward against a central difference of the GPU misfit (FP64
    accumulated) along a smooth direction.  The traces are FP32, so the difference is
    taken over a 1 % velocity change and agreement is checked to 1e-2 (the strict FD pin
    of the gradient, 1e-6, is the oracle's; the GPU gradient matches the oracle to 1e-3)."""
    f = fwi()
    rng = np.random.default_rng(31)
    w, dobs = _grad_case(2, (36, 44), 8, nt=120)
    w.src[0, 2] = 20
    m, _, acq = make_pair(w, snap="fp32")
    wav = torch.from_numpy(w.wavelets()).cuda()
    d = torch.from_numpy(dobs).cuda()
    v = torch.from_numpy(w.v).cuda().requires_grad_(True)
    phi = f.WaveFwi.apply(v, m, acq, wav, d)
    phi.backward()
    dv = torch.from_numpy(50.0 * synth.gaussian_random_field(rng, w.v.shape, w.h, 80.0, 1.0)).cuda()
    eps = 0.6   # 30 m/s along dv: about 1 % of the velocity
    fp = f.WaveFwi.apply((v + eps * dv).detach(), m, acq, wav, d).item()
    fm = f.WaveFwi.apply((v - eps * dv).detach(), m, acq, wav, d).item()
    fd = (fp - fm) / (2 * eps)
    an = float(torch.sum(v.grad.double() * dv.double()))
    print(f"autograd FD: fd {fd:.6e} adjoint {an:.6e} rel {abs(fd - an) / abs(an):.2e}")
    assert abs(fd - an) <= 1e-2 * abs(an)


@pytest.mark.parametrize("snap", ["bf16", "fp16"])
@pytest.mark.parametrize("ndim,shape,order", [(2, (40, 52), 8), (3, (15, 16, 18), 16)])
def test_gradient_16bit_checkpoints(snap, ndim, shape, order):
    w, dobs = _grad_case(ndim, shape, order, nt=90, f0=10.0)
    probe, _, _ = make_pair(w, snap=snap, budget=1)
    pitch, comp = probe.info()["pitch_x"], probe.info()["computed"]
    field = -(-comp[0] * comp[1] * pitch // 64) * 64
    m, p, acq = make_pair(w, snap=snap, budget=8 * 2 * 2 * field)   # eight checkpoints
    _, g = m.gradient(acq, torch.from_numpy(w.wavelets()).cuda(), torch.from_numpy(dobs).cuda())
    info = m.info()
    assert 0 < info["snap_slots"] < w.nt    # recomputation really happened
    rphi, rg = p.gradient(dobs.astype(np.float64))
    e = rel(g.cpu().numpy(), rg)
    print(f"grad {snap} {ndim}d: rel-L2 {e:.2e} slots {info['snap_slots']}")
    assert e <= TOL_GRAD16


# ------------------------------------------------------------------ errors

def test_errors_are_reported():
    f = fwi()
    rng = np.random.default_rng(3)
    w = synth.random_small(rng, 2, (20, 20), nt=10, nb=3)
    with pytest.raises(f.FwiError) as e:
        f.FwiModel(torch.from_numpy(w.v).cuda(), w.h, w.dt * 3.0, w.nt, nb=3)
    assert e.value.code == f.FWI_ERR_CFL
    m, _, _ = make_pair(w)
    bad = f.Acquisition([[25, 0, 3]], w.rec)
    with pytest.raises(f.FwiError) as e:
        m.forward(bad, torch.from_numpy(w.wavelets()).cuda())
    assert e.value.code == f.FWI_ERR_ARG
    # a host-poisoned wavelet drives the wavefield non-finite: latched and reported
    wav = w.wavelets().copy()
    wav[0, 2] = np.inf
    acq = f.Acquisition(w.src, w.rec)
    m.forward(acq, torch.from_numpy(wav).cuda())
    with pytest.raises(f.FwiError) as e:
        f.fwi_sync_status(m.handle)
    assert e.value.code == f.FWI_ERR_UNSTABLE


@pytest.mark.parametrize("snap", ["bf16", "fp32"])
@pytest.mark.parametrize("ndim,shape,order", [(2, (40, 52), 8), (3, (15, 16, 18), 16)])
def test_gradient_store_all_half_slots(snap, ndim, shape, order):
    """A budget that holds u^n alone for every step but not pairs: the schedule runs the
    forward recursion once (nt forward steps, nt - 1 checkpoints, each restored only for
    its reverse step), in slots of half the pair size; the gradient meets the same bars
    as with recomputation, and with FP32 checkpoints equals the recomputing run's."""
    w, dobs = _grad_case(ndim, shape, order, nt=90, f0=10.0)
    probe, _, _ = make_pair(w, snap=snap, budget=1)
    pitch, comp = probe.info()["pitch_x"], probe.info()["computed"]
    field = -(-comp[0] * comp[1] * pitch // 64) * 64
    esz = 4 if snap == "fp32" else 2
    m, p, acq = make_pair(w, snap=snap, budget=(w.nt - 1) * field * esz)
    wav, d = torch.from_numpy(w.wavelets()).cuda(), torch.from_numpy(dobs).cuda()
    _, g = m.gradient(acq, wav, d)
    info = m.info()
    assert info["snap_slots"] == w.nt - 1 and info["last_forward_steps"] == w.nt
    rphi, rg = p.gradient(dobs.astype(np.float64))
    e = rel(g.cpu().numpy(), rg)
    print(f"store-all grad {snap} {ndim}d: rel-L2 {e:.2e}")
    assert e <= (TOL_GRAD32 if snap == "fp32" else TOL_GRAD16)
    if snap == "fp32":
        m2, _, _ = make_pair(w, snap=snap, budget=8 * 2 * esz * field)
        _, g2 = m2.gradient(acq, wav, d)
        assert m2.info()["last_forward_steps"] > w.nt
        assert torch.equal(g, g2)


@pytest.mark.parametrize("order", [8, 16])
def test_anisotropic_spacing_3d(order):
    """hz, hy, hx all different: the 3-D step takes its per-axis weights from the launch
    parameters (an isotropic grid runs the instantiation with compile-time weights, which
    every other 3-D test exercises); traces and the FP32-checkpoint gradient against the
    oracle at the usual bars."""
    rng = np.random.default_rng(40 + order)
    h = (10.0, 12.5, 8.0)
    w = synth.random_small(rng, 3, (14, 15, 17), h=10.0, nt=60, order=order, nb=5, nrec=9)
    w.h = h
    w.dt = 0.4 * min(h) / 4500.0
    vobs = w.v * (0.92 + 0.04 * synth.gaussian_random_field(rng, w.v.shape, 10.0, 40.0, 1.0))
    p_obs = oracle.Problem(vobs, h, w.dt, w.nt, order=order, nb=5, vref=4600.0, src=w.src,
                           rec=w.rec, wavelet=w.wavelets())
    dobs = p_obs.forward().astype(np.float32)
    m, p, acq = make_pair(w, snap="fp32")
    wav = torch.from_numpy(w.wavelets()).cuda()
    tr = m.forward(acq, wav).cpu().numpy()
    e_tr = rel(tr, p.forward())
    _, g = m.gradient(acq, wav, torch.from_numpy(dobs).cuda())
    e_g = rel(g.cpu().numpy(), p.gradient(dobs.astype(np.float64))[1])
    print(f"anisotropic 3-D o{order}: traces {e_tr:.2e}, gradient {e_g:.2e}")
    assert e_tr <= TOL_FWD and e_g <= TOL_GRAD32


def test_model_reuse_across_checkpoint_layouts():
    """One model, one budget, calls whose checkpoint layouts differ: 1 shot fits u^n of
    every step (store-all, one field per slot), 2 shots do not (recomputation, pair slots
    among them).  The pool is re-zeroed when its layout changes, so every call equals the
    same call on a fresh model bit for bit."""
    w, dobs = _grad_case(2, (40, 52), 8, nt=90, f0=10.0, nshots=2)
    probe, _, _ = make_pair(w, snap="bf16", budget=1)
    pitch, comp = probe.info()["pitch_x"], probe.info()["computed"]
    field = -(-comp[0] * comp[1] * pitch // 64) * 64
    budget = (w.nt - 1) * field * 2
    f = fwi()
    wav = torch.from_numpy(w.wavelets()).cuda()
    d = torch.from_numpy(dobs).cuda()
    acq2 = f.Acquisition(w.src, w.rec)
    acq1 = f.Acquisition(w.src[:1], w.rec)

    def fresh(acq, ns):
        m, _, _ = make_pair(w, snap="bf16", budget=budget)
        return m.gradient(acq, wav[:ns], d[:ns])[1]

    m, _, _ = make_pair(w, snap="bf16", budget=budget)
    g1a = m.gradient(acq1, wav[:1], d[:1])[1]
    assert m.info()["last_forward_steps"] == w.nt          # store-all
    g2 = m.gradient(acq2, wav, d)[1]
    assert m.info()["last_forward_steps"] > w.nt           # recomputation
    g1b = m.gradient(acq1, wav[:1], d[:1])[1]
    assert torch.equal(g1a, g1b)
    assert torch.equal(g1a, fresh(acq1, 1)) and torch.equal(g2, fresh(acq2, 2))


@pytest.mark.parametrize("order", [16, 8])
@pytest.mark.parametrize("tmem,tile_g,half",
                         [("1", "0", "1"), ("1", "1", "0"), ("1", "0", "0"), ("0", "0", "0")])
def test_step_kernels_both_variants(tmem, tile_g, half, order, monkeypatch):
    """The 3-D steps run either the tensor-memory kernel (z-stream in TMEM; FWI_STEP3D_TMEM=1),
    with its forward modes on 64 x 16 tiles of 4 warps or 64 x 32 tiles of 8 warps
    (FWI_STEP3D_HALF=1/0) and its reverse step staging g per thread or reading it as a TMA
    tile (FWI_STEP3D_TILE_G=0/1), or the register-queue kernel (FWI_STEP3D_TMEM=0), at
    radius 8 and radius 4; every combination matches the oracle in every mode: forward,
    forward with checkpoint stores, reverse step with imaging (FP16 checkpoints,
    recomputation)."""
    monkeypatch.setenv("FWI_STEP3D_TMEM", tmem)
    monkeypatch.setenv("FWI_STEP3D_TILE_G", tile_g)
    monkeypatch.setenv("FWI_STEP3D_HALF", half)
    rng = np.random.default_rng(31)
    w = synth.random_small(rng, 3, (22, 37, 70), nt=70, order=order, nb=4, nrec=9)
    m, p, acq = make_pair(w, snap="fp16", budget=1)
    probe = m.info()
    field = probe["computed"][0] * probe["computed"][1] * probe["pitch_x"]
    m.close()
    m, p, acq = make_pair(w, snap="fp16", budget=6 * 2 * 2 * (-(-field // 64) * 64))
    wav = torch.from_numpy(w.wavelets()).cuda()
    tr = m.forward(acq, wav).cpu().numpy()
    ref = p.forward()
    et = rel(tr, ref)
    dobs = (ref * 0.8).astype(np.float32)
    phi, g = m.gradient(acq, wav, torch.from_numpy(dobs).cuda())
    info = m.info()
    rphi, rg = p.gradient(dobs.astype(np.float64))
    eg = rel(g.cpu().numpy(), rg)
    print(f"order {order}, TMEM {tmem}, tile g {tile_g}, half {half}: traces {et:.2e}, gradient {eg:.2e}, "
          f"slots {info['snap_slots']}, forward steps {info['last_forward_steps']}")
    assert 0 < info["snap_slots"] < w.nt
    assert et <= TOL_FWD and eg <= TOL_GRAD16
    assert abs(phi.item() - rphi) <= TOL_GRAD32 * rphi


@pytest.mark.parametrize("order", [16, 8])
def test_reverse_step_forms_are_bit_equal(order, monkeypatch):
    """The tensor-memory reverse step's two ways of reading g (per-thread asynchronous
    copies into a staging buffer, or a TMA pointwise tile) do the same arithmetic in the
    same order: gradients equal bit for bit, on a grid whose ragged tiles leave rows and
    columns outside the field."""
    monkeypatch.setenv("FWI_STEP3D_TMEM", "1")
    rng = np.random.default_rng(35)
    w = synth.random_small(rng, 3, (29, 41, 67), nt=40, order=order, nb=4, nrec=7)
    wav = torch.from_numpy(w.wavelets()).cuda()
    m, p, acq = make_pair(w, snap="fp16")
    dobs = torch.from_numpy((p.forward() * 0.8).astype(np.float32)).cuda()
    out = {}
    for tg in ("0", "1"):
        monkeypatch.setenv("FWI_STEP3D_TILE_G", tg)
        out[tg] = m.gradient(acq, wav, dobs)
    assert torch.equal(out["0"][1], out["1"][1])
    assert out["0"][0].item() == out["1"][0].item()


def test_gradient_from_host_buffers():
    """Wavelets, d_obs and the outputs in host memory, pageable (numpy) and pinned (torch):
    the library stages them itself.  Misfit and gradient equal those of device inputs bit
    for bit, and match the oracle."""
    f = fwi()
    rng = np.random.default_rng(37)
    w = synth.random_small(rng, 3, (24, 30, 40), nt=60, order=16, nb=4, nrec=9)
    m, p, acq = make_pair(w, snap="fp16")
    wav = np.ascontiguousarray(w.wavelets(), dtype=np.float32)
    ref = p.forward()
    dobs = np.ascontiguousarray(ref * 0.8, dtype=np.float32)
    phi_d, g_d = m.gradient(acq, torch.from_numpy(wav).cuda(), torch.from_numpy(dobs).cuda())
    g_d = g_d.cpu().numpy()
    rphi, rg = p.gradient(dobs.astype(np.float64))
    for pinned in (False, True):
        if pinned:
            wav_h = torch.from_numpy(wav).pin_memory()
            dobs_h = torch.from_numpy(dobs).pin_memory()
            grad_h = torch.empty(g_d.shape, dtype=torch.float32).pin_memory()
        else:
            wav_h, dobs_h = wav.copy(), dobs.copy()
            grad_h = np.empty(g_d.shape, dtype=np.float32)
        phi_h = np.zeros(1, dtype=np.float64)
        f.fwi_adjoint_gradient(m.handle, acq.c, wav_h, dobs_h, phi_h, grad_h)
        g_h = grad_h.numpy() if pinned else grad_h
        assert phi_h[0] == phi_d.item()
        assert np.array_equal(g_h, g_d)
        assert rel(g_h, rg) <= TOL_GRAD16 and abs(phi_h[0] - rphi) <= TOL_GRAD32 * rphi


def test_2d_batch_with_l2_prefetch_equals_single_shots():
    """A 2-D batch whose fields exceed 96 MB (64 shots of the faulted model, 440 x 1064
    computed points, 120 MB per field) runs its steps with the streamed rows prefetched
    into L2; one-shot calls of the same shots run without.  The prefetches change no
    arithmetic: the traces equal bit for bit, and the batch's FP64 gradient equals the sum
    of the one-shot FP64 gradients to rounding."""
    f = fwi()
    w = synth.faulted_2d(nt=120)
    acq = f.Acquisition(w.src, w.rec)
    wav = torch.from_numpy(np.ascontiguousarray(w.wavelets())).cuda()
    m = f.FwiModel(torch.from_numpy(np.ascontiguousarray(w.v)).cuda(), w.h, w.dt, w.nt,
                   order=w.order, snap_dtype="fp32", sponge_vref=4500.0)
    tr = m.forward(acq, wav)
    dobs = (tr * 0.9).contiguous()
    _, _, g64 = m.gradient(acq, wav, dobs, want64=True)
    gsum = torch.zeros_like(g64)
    for i in range(w.nshots):
        one = f.Acquisition(w.src[i:i + 1], w.rec)
        if i in (0, w.nshots // 2, w.nshots - 1):
            assert torch.equal(m.forward(one, wav[i:i + 1])[0], tr[i])
        gsum += m.gradient(one, wav[i:i + 1], dobs[i:i + 1], want64=True)[2]
    e = ((g64 - gsum).norm() / gsum.norm()).item()
    print(f"64-shot 2-D batch against one-shot calls: gradient rel-L2 {e:.2e}")
    assert e <= 1e-10
    m.close()


@pytest.mark.parametrize("tma", ["1", "0"])
def test_2d_step_kernels_both_variants(tma, monkeypatch):
    """The 2-D step runs either the register-streaming kernel (default) or the TMA-staged
    one (FWI_STEP2D_TMA=1); traces and FP32-checkpoint gradients equal each other bit for
    bit and match the oracle, for a batch of shots at orders 8 and 16."""
    monkeypatch.setenv("FWI_STEP2D_TMA", tma)
    rng = np.random.default_rng(33)
    for order in (8, 16):
        w = synth.random_small(rng, 2, (61, 300), nt=90, order=order, nb=6, nrec=11)
        m, p, acq = make_pair(w, snap="fp32")
        wav = torch.from_numpy(w.wavelets()).cuda()
        tr = m.forward(acq, wav).cpu().numpy()
        ref = p.forward()
        dobs = (ref * 0.8).astype(np.float32)
        phi, g = m.gradient(acq, wav, torch.from_numpy(dobs).cuda())
        rphi, rg = p.gradient(dobs.astype(np.float64))
        et, eg = rel(tr, ref), rel(g.cpu().numpy(), rg)
        print(f"2-D order {order}, TMA {tma}: traces {et:.2e}, gradient {eg:.2e}")
        assert et <= TOL_FWD and eg <= TOL_GRAD32


@pytest.mark.parametrize("order", [8, 16])
def test_receivers_fused_into_the_3d_steps(order, monkeypatch):
    """Node receivers on one plane: the 3-D forward steps sample them and the reverse
    steps inject the residual in their epilogues (no separate launches).  Traces, misfit
    and gradient equal the separate-kernel path (FWI_STEP3D_REC_FUSE=0) bit for bit and
    match the oracle; two shots with different receiver lines, FP16 checkpoints with
    recomputation."""
    rng = np.random.default_rng(35 + order)
    w = synth.random_small(rng, 3, (26, 33, 47), nt=60, order=order, nb=4, nrec=1)
    w.src = np.array([[3, 10, 20], [4, 25, 30]], dtype=np.int32)
    w.rec = np.array([[[2, y, x] for y in range(1, 33, 3) for x in range(0, 47, 2)],
                      [[2, y, x] for y in range(0, 33, 3) for x in range(0, 47, 2)]],
                     dtype=np.int32)
    outs = []
    for fuse in ("1", "0"):
        monkeypatch.setenv("FWI_STEP3D_REC_FUSE", fuse)
        m, p, acq = make_pair(w, snap="fp16", budget=1)
        probe = m.info()
        field = probe["computed"][0] * probe["computed"][1] * probe["pitch_x"]
        m.close()
        m, p, acq = make_pair(w, snap="fp16", budget=2 * 5 * 2 * 2 * (-(-field // 64) * 64))
        wav = torch.from_numpy(w.wavelets()).cuda()
        tr = m.forward(acq, wav).cpu().numpy()
        dobs = (p.forward() * 0.7).astype(np.float32)
        phi, g = m.gradient(acq, wav, torch.from_numpy(dobs).cuda())
        info = m.info()
        m.close()
        outs.append((tr, phi.item(), g.cpu().numpy(), info))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1] and np.array_equal(outs[0][2], outs[1][2])
    assert 0 < outs[0][3]["snap_slots"] < w.nt
    # the fused run launched fewer kernels (no per-step sampling or injection)
    assert outs[0][3]["kernel_launches"] < outs[1][3]["kernel_launches"]
    ref = p.forward()
    rphi, rg = p.gradient(dobs.astype(np.float64))
    et, eg = rel(outs[0][0], ref), rel(outs[0][2], rg)
    print(f"fused receivers order {order}: traces {et:.2e}, gradient {eg:.2e}")
    assert et <= TOL_FWD and eg <= TOL_GRAD16
