"""Serving loop (continuous batching): each request's result is the same alone and in
the mix, work from several requests overlaps, and admission respects the memory budget."""
import math

import numpy as np
import pytest

from paper_1912_08063_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _requests(n, seed):
    from paper_1912_08063_gb300 import fwi

    def dt_for(ndim, h):
        lim = 1.0 / fwi.fwi_cfl_number(ndim, 8, (h, h, h), 4500.0, 1.0)
        return math.floor(0.8 * lim * 1e4) / 1e4

    reqs = synth.serving_requests(n, dt_for, seed=seed, size2d=(40, 140), size3d=(20, 44),
                                  nt_range=(60, 220))
    for r in reqs:
        if r["kind"] == "gradient":   # observed traces from the perturbed model
            m = fwi.FwiModel(torch.from_numpy(r["v_obs"]).cuda(), r["h"], r["dt"], r["nt"])
            acq = fwi.Acquisition([r["src"]], r["rec"])
            r["d_obs"] = m.forward(acq, torch.from_numpy(r["wavelet"][None]).cuda())[0].cpu().numpy()
            m.close()
    return reqs


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_results_same_alone_and_in_the_mix():
    from paper_1912_08063_gb300 import fwi
    reqs = _requests(8, seed=1)
    for i, r in enumerate(reqs):
        r["arrival"] = 0.002 * i
    mix, mix_out = fwi.fwi_serve(reqs, max_active=8, steps_per_turn=4, snap_slots=6)
    assert all(x["status"] == 0 for x in mix), mix
    for i, r in enumerate(reqs):
        r1 = dict(r, arrival=0.0)
        alone, alone_out = fwi.fwi_serve([r1], max_active=1, snap_slots=6)
        assert alone[0]["status"] == 0
        e = _rel(mix_out[i], alone_out[0])
        assert e <= 1e-6, (i, r["kind"], e)
        if r["kind"] == "gradient":
            assert abs(mix[i]["misfit"] - alone[0]["misfit"]) <= 1e-6 * abs(alone[0]["misfit"])
            assert np.abs(alone_out[0]).max() > 0
    # the requests really ran together: some [start, done] intervals overlap
    iv = sorted((x["t_start"], x["t_done"]) for x in mix)
    assert any(b[0] < a[1] for a, b in zip(iv, iv[1:]))


def test_admission_respects_the_budget():
    from paper_1912_08063_gb300 import fwi
    reqs = _requests(10, seed=2)
    # a budget that holds only a few of these requests at once
    budget = 3 * 10 ** 8
    res, _ = fwi.fwi_serve(reqs, budget_bytes=budget, max_active=16, steps_per_turn=4,
                           snap_slots=4)
    assert all(x["status"] == 0 for x in res), res
    for x in res:
        assert 0 < x["device_bytes"] <= x["reserved_bytes"], x
    events = sorted([(x["t_admit"], x["reserved_bytes"]) for x in res] +
                    [(x["t_done"], -x["reserved_bytes"]) for x in res], key=lambda e: (e[0], e[1]))
    held = 0
    for _, d in events:
        held += d
        assert held <= budget
    # and requests were admitted as memory freed up, not all at once
    assert len({round(x["t_admit"], 6) for x in res}) > 1


@pytest.mark.parametrize("shared", [True, False])
def test_graph_replayed_forward_equals_direct_call(shared):
    """Forward requests in the serving loop run either in the shared launch (2-D: one
    graph per tick of multi-request step and sampling kernels over a table of request
    descriptors) or, without it, as per-request turns replayed from captured CUDA graphs
    that read the step index from a device counter (turns of 6 steps here; nt not a
    multiple of 6, so the last steps run one by one); either way the traces equal a direct
    forward call bit for bit."""
    from paper_1912_08063_gb300 import fwi
    reqs = [r for r in _requests(10, seed=5) if r["kind"] == "forward"][:4]
    assert reqs
    for r in reqs:
        r["arrival"] = 0.0
    res, out = fwi.fwi_serve(reqs, max_active=4, steps_per_turn=6, snap_slots=4,
                             shared_launch=shared)
    n2d = sum(1 for r in reqs if r["v"].ndim == 2)
    assert sum(1 for x in res if x["shared_launch"]) == (n2d if shared else 0)
    for r, x, o in zip(reqs, res, out):
        assert x["status"] == 0
        m = fwi.FwiModel(torch.from_numpy(r["v"]).cuda(), r["h"], r["dt"], r["nt"])
        acq = fwi.Acquisition([r["src"]], r["rec"])
        direct = m.forward(acq, torch.from_numpy(r["wavelet"][None]).cuda())[0].cpu().numpy()
        m.close()
        assert np.array_equal(np.asarray(o).reshape(direct.shape), direct)


def test_graph_replayed_gradient_equals_direct_call():
    """Gradient requests replay runs of plain forward steps as CUDA graphs in turns of 16
    steps; with the same checkpoint budget the gradient and misfit equal a direct call
    (steps issued one by one) bit for bit."""
    from paper_1912_08063_gb300 import fwi
    reqs = [r for r in _requests(12, seed=6) if r["kind"] == "gradient"][:3]
    assert reqs
    for r in reqs:
        r["arrival"] = 0.0
    slots = 5
    res, out = fwi.fwi_serve(reqs, max_active=3, steps_per_turn=16, snap_slots=slots)
    for r, x, o in zip(reqs, res, out):
        assert x["status"] == 0
        shp = r["v"].shape
        nz = shp[0] + 40
        ny = shp[1] + 40 if len(shp) == 3 else 1
        nx = shp[-1] + 40
        field = -(-(nz * ny * (-(-nx // 8) * 8)) // 64) * 64
        m = fwi.FwiModel(torch.from_numpy(r["v"]).cuda(), r["h"], r["dt"], r["nt"],
                         snap_dtype=r["snap_dtype"], snap_budget_bytes=slots * 2 * field * 2)
        acq = fwi.Acquisition([r["src"]], r["rec"])
        phi, g = m.gradient(acq, torch.from_numpy(r["wavelet"][None]).cuda(),
                            torch.from_numpy(r["d_obs"][None]).cuda())
        m.close()
        assert x["misfit"] == phi.item()
        assert np.array_equal(np.asarray(o).reshape(g.shape), g.cpu().numpy())


def test_served_results_match_the_oracle():
    """One forward and one gradient request served in a mix with others, against the FP64
    oracle on the same inputs: traces to 1e-4 and the BF16-checkpoint gradient to 1e-2
    (relative L2), as for direct calls.  The observed traces of the gradient request come
    from the oracle's forward run of the perturbed model."""
    import oracle
    from paper_1912_08063_gb300 import fwi
    reqs = _requests(8, seed=11)
    # a 2-D forward request (it runs in the shared launch) and a gradient request
    fwd = next(i for i, r in enumerate(reqs) if r["kind"] == "forward" and r["v"].ndim == 2)
    grd = next(i for i, r in enumerate(reqs) if r["kind"] == "gradient")

    def problem(r, v):
        return oracle.Problem(v, r["h"], r["dt"], r["nt"], order=8, nb=20,
                              src=np.asarray(r["src"])[None], rec=r["rec"],
                              wavelet=r["wavelet"][None])

    rg = reqs[grd]
    rg["d_obs"] = problem(rg, rg["v_obs"]).forward()[0].astype(np.float32)
    for i, r in enumerate(reqs):
        r["arrival"] = 0.001 * i
    res, out = fwi.fwi_serve(reqs, max_active=8, steps_per_turn=4, snap_slots=6)
    assert all(x["status"] == 0 for x in res), res
    assert res[fwd]["shared_launch"] > 0 and res[grd]["shared_launch"] == 0
    rf = reqs[fwd]
    ref = problem(rf, rf["v"]).forward()[0]
    e = _rel(np.asarray(out[fwd]).reshape(ref.shape), ref)
    print(f"served forward ({rf['v'].ndim}-D {rf['v'].shape}, nt {rf['nt']}): rel-L2 {e:.2e}")
    assert e <= 1e-4
    phi, g = problem(rg, rg["v"]).gradient(rg["d_obs"][None].astype(np.float64))
    eg = _rel(np.asarray(out[grd]).reshape(g.shape), g)
    ephi = abs(res[grd]["misfit"] - phi) / phi
    print(f"served gradient ({rg['v'].ndim}-D {rg['v'].shape}, nt {rg['nt']}, "
          f"{rg['snap_dtype']}): rel-L2 {eg:.2e}, misfit {ephi:.2e}")
    assert eg <= 1e-2 and ephi <= 1e-4


def test_shared_launch_equals_own_streams():
    """A mixed stream served with the shared launch and without it: every result is the
    same bit for bit (the shared launch runs the same step arithmetic), the 2-D forward
    requests ran in the shared launch, and several of them were in it at once."""
    from paper_1912_08063_gb300 import fwi
    reqs = _requests(12, seed=7)
    for r in reqs:
        r["arrival"] = 0.0
    a, oa = fwi.fwi_serve(reqs, max_active=12, steps_per_turn=4, snap_slots=6)
    b, ob = fwi.fwi_serve(reqs, max_active=12, steps_per_turn=4, snap_slots=6,
                          shared_launch=False)
    assert all(x["status"] == 0 for x in a + b)
    pooled = [i for i, r in enumerate(reqs) if r["kind"] == "forward" and r["v"].ndim == 2]
    assert len(pooled) >= 2
    assert [i for i, x in enumerate(a) if x["shared_launch"]] == pooled
    assert not any(x["shared_launch"] for x in b)
    for i in range(len(reqs)):
        assert np.array_equal(oa[i], ob[i]), i
        assert a[i]["misfit"] == b[i]["misfit"]
    iv = sorted((a[i]["t_start"], a[i]["t_done"]) for i in pooled)
    assert any(y[0] < x[1] for x, y in zip(iv, iv[1:]))


def test_cluster_launch_small_and_large_requests():
    """Small 2-D forward requests run in the cluster launch (k steps per launch, both
    states in the shared memory of one cluster), larger ones in the multi-request step
    launch; both equal direct forward calls bit for bit, and one of each matches the
    oracle."""
    import oracle
    from paper_1912_08063_gb300 import fwi

    def dt_for(ndim, h):
        lim = 1.0 / fwi.fwi_cfl_number(ndim, 8, (h, h, h), 4500.0, 1.0)
        return math.floor(0.8 * lim * 1e4) / 1e4

    reqs = synth.serving_requests(40, dt_for, seed=9, size2d=(40, 900), size3d=(20, 24),
                                  nt_range=(30, 90), frac_grad=0.0, frac_2d=1.0)
    for r in reqs:
        r["arrival"] = 0.0
    res, out = fwi.fwi_serve(reqs, max_active=16, steps_per_turn=8, snap_slots=4)
    kinds = [x["shared_launch"] for x in res]
    assert all(x["status"] == 0 for x in res) and 1 in kinds and 2 in kinds, kinds
    for r, x, o in zip(reqs, res, out):
        m = fwi.FwiModel(torch.from_numpy(r["v"]).cuda(), r["h"], r["dt"], r["nt"])
        acq = fwi.Acquisition([r["src"]], r["rec"])
        direct = m.forward(acq, torch.from_numpy(r["wavelet"][None]).cuda())[0].cpu().numpy()
        m.close()
        assert np.array_equal(np.asarray(o).reshape(direct.shape), direct), x["shared_launch"]
    for kind in (1, 2):
        i = min((j for j, k in enumerate(kinds) if k == kind), key=lambda j: reqs[j]["v"].size)
        r = reqs[i]
        ref = oracle.Problem(r["v"], r["h"], r["dt"], r["nt"], order=8, nb=20,
                             src=np.asarray(r["src"])[None], rec=r["rec"],
                             wavelet=r["wavelet"][None]).forward()[0]
        e = _rel(np.asarray(out[i]).reshape(ref.shape), ref)
        print(f"shared launch kind {kind}, {r['v'].shape}: traces rel-L2 {e:.2e}")
        assert e <= 1e-4
