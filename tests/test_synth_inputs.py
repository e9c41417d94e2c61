"""The seeded synthetic inputs follow the stated recipe (shapes, value ranges, geometry,
seeding), independently of the solvers: config 1's two-layer model, config 2's layered
model with random perturbations, config 3's faulted model with a salt ellipse and its
64 evenly spaced shots, config 5's salt model and its twins, the serving request mix,
the Ricker wavelet and the Gaussian random field."""
import numpy as np
import pytest

from paper_1912_08063_gb300 import synth


def test_two_layer_config1():
    w = synth.two_layer_2d()
    assert w.shape == (201, 201) and w.nt == 500 and w.dt == 1e-3 and w.h == 10.0
    assert np.all(w.v[:100] == 1500.0) and np.all(w.v[100:] == 2500.0)
    assert w.src.tolist() == [[10, 0, 100]]
    assert w.nrec == 201 and np.all(w.rec[:, 0] == 5) and w.rec[:, 2].tolist() == list(range(201))
    assert w.order == 8 and w.f0 == 15.0


def test_ricker_peak_and_zero_mean():
    f0, dt, nt = 15.0, 1e-4, 4000
    r = synth.ricker(f0, dt, nt)
    t = np.arange(nt) * dt
    assert t[np.argmax(r)] == pytest.approx(1.5 / f0, abs=dt)
    assert r.max() == pytest.approx(1.0, abs=1e-6)
    assert abs(r.sum() * dt) < 1e-6           # the Ricker wavelet integrates to zero


def test_gaussian_random_field_normalised():
    rng = np.random.default_rng(0)
    f = synth.gaussian_random_field(rng, (64, 80), 10.0, 200.0, 0.05)
    assert abs(float(f.mean())) < 1e-6 and float(f.std()) == pytest.approx(0.05, rel=1e-4)
    # correlated over ~ell: neighbouring cells nearly equal, far cells much less so
    c1 = np.corrcoef(f[:, :-1].ravel(), f[:, 1:].ravel())[0, 1]
    c40 = np.corrcoef(f[:, :-40].ravel(), f[:, 40:].ravel())[0, 1]
    assert c1 > 0.95 and c40 < c1 - 0.3


@pytest.mark.parametrize("make", [lambda: synth.faulted_2d(nz=100, nx=256, nt=10, nshots=8),
                                  lambda: synth.layered_3d(24, nt=10),
                                  lambda: synth.salt_3d(32, nt=64)])
def test_seeded_and_reproducible(make):
    a, b = make(), make()
    assert np.array_equal(a.v, b.v) and np.array_equal(a.src, b.src)
    assert np.array_equal(a.rec, b.rec)
    if a.v_obs is not None:
        assert np.array_equal(a.v_obs, b.v_obs) and not np.array_equal(a.v, a.v_obs)


def test_faulted_2d_config3():
    w = synth.faulted_2d(nt=10)
    assert w.shape == (400, 1024) and w.nshots == 64 and w.nrec == 1024
    assert w.order == 8 and w.f0 == 20.0 and w.dt == 1e-3 and w.snap_dtype == "bf16"
    assert w.src[:, 2].tolist() == [8 + 16 * i for i in range(64)]    # evenly spaced
    assert np.all(w.src[:, 0] == 10) and np.all(w.rec[:, 0] == 5)
    for v in (w.v, w.v_obs):
        assert v.dtype == np.float32 and v.min() >= 1500.0 and v.max() <= 4500.0
    salt = w.v == 4500.0
    assert 0.005 < salt.mean() < 0.2                 # an ellipse of the stated size
    # the perturbed model differs by about 5 % outside the clip
    rel = (w.v_obs / w.v - 1.0)[~salt]
    assert 0.02 < float(rel.std()) < 0.08


def test_layered_3d_config2():
    w = synth.layered_3d(48, nt=10)
    assert w.shape == (48, 48, 48) and w.order == 8 and w.snap_dtype == "bf16"
    assert w.src.tolist() == [[10, 24, 24]] and np.all(w.rec[:, 0] == 5)
    assert w.v.min() >= 1500.0 and w.v.max() <= 4500.0
    # layered: the horizontal mean velocity grows with depth, top to bottom
    mz = w.v.mean(axis=(1, 2))
    assert mz[-1] > mz[0] + 1000.0


def test_salt_3d_twin_scaling():
    w = synth.salt_3d(64)
    assert w.shape == (64, 64, 64) and w.order == 16 and w.snap_dtype == "fp16"
    assert w.h == pytest.approx(12.5 * 512 / 64) and w.dt == pytest.approx(0.6e-3 * 512 / 64)
    assert w.nt == 500 and w.f0 == pytest.approx(15.0 * 64 / 512)
    assert np.any(w.v == 4500.0) and w.v.min() >= 1500.0
    assert w.nrec == 32 * 32                          # every 2nd cell of the surface row


def test_serving_request_mix():
    reqs = synth.serving_requests(200, lambda ndim, h: 1e-3)
    two_d = [r for r in reqs if r["v"].ndim == 2]
    assert 0.6 < len(two_d) / len(reqs) < 0.9
    assert 0.35 < sum(r["kind"] == "gradient" for r in reqs) / len(reqs) < 0.65
    for r in reqs:
        assert 500 <= r["nt"] <= 3000 and r["order"] == 8 and r["snap_dtype"] == "bf16"
        lo, hi = (128, 1024) if r["v"].ndim == 2 else (64, 192)
        assert all(lo <= s <= hi for s in r["v"].shape)
        assert r["v"].min() >= 1500.0 - 1e-3 and r["v"].max() <= 4500.0 + 1e-3
        assert ("v_obs" in r) == (r["kind"] == "gradient")
