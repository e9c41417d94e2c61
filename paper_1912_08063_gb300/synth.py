"""Seeded synthetic inputs: velocity models, source wavelets and acquisition geometry.

This module holds none of the method's arithmetic (no stencil, no time stepping, no
adjoint): it only draws the inputs that both the CUDA path and the FP64 oracle are fed.
All randomness comes from ``numpy.random.Generator(PCG64(19_120_8063 + config id))``.

Workloads (sizes are physical grids; the sponge of ``nb`` cells is added by the solver):

* ``two_layer_2d``      201 x 201 (z, x), h = 10 m, dt = 1 ms, nt = 500, 8th order,
                        1500 / 2500 m/s split at row 100, 15 Hz Ricker at (iz 10, ix 100),
                        201 receivers on row 5.
* ``layered_3d``        256^3, h = 10 m, dt = 0.8 ms, nt = 2000, 8th order, 8 layers
                        1500 -> 4500 m/s with +-100 m/s jitter times (1 + delta), delta a
                        Gaussian random field (std 5 %, correlation length 200 m);
                        128 x 128 receivers every 2nd cell on row 5; observed data from an
                        independently perturbed model.  ``scale`` gives the 64^3 instance.
* ``faulted_2d``        400 x 1024 (z, x), h = 10 m, dt = 1 ms, nt = 3000, 8th order,
                        6 layers 1500 -> 3500 m/s, 3 dipping faults, a 4500 m/s salt
                        ellipse, 64 shots at ix = 8 + 16 i, 1024 receivers, 20 Hz Ricker.
* ``salt_3d``           512^3, h = 12.5 m, dt = 0.6 ms, nt = 4000, 16th order, 10 layers
                        1500 -> 4500 m/s, 3 dipping fault planes, a 4500 m/s salt
                        ellipsoid, 256 x 256 receivers every 2nd cell; ``scale`` gives the
                        96^3 twin (h scaled so the physical size is kept).
* ``smooth_random``     serving requests: 2-D or 3-D smooth random fields mapped to
                        1500..4500 m/s.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

SEED_BASE = 1912_08063


def rng_for(config_id: int, extra: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + config_id + extra))


def ricker(f0: float, dt: float, nt: int, t0: Optional[float] = None) -> np.ndarray:
    """Ricker wavelet sampled at t = n dt (FP64 on the host, returned as FP32):
    (1 - 2 pi^2 f^2 (t - t0)^2) exp(-pi^2 f^2 (t - t0)^2), t0 = 1.5 / f by default."""
    t0 = 1.5 / f0 if t0 is None else t0
    t = np.arange(nt, dtype=np.float64) * dt - t0
    a = (math.pi * f0 * t) ** 2
    return ((1.0 - 2.0 * a) * np.exp(-a)).astype(np.float32)


def _upsample_linear(a: np.ndarray, shape) -> np.ndarray:
    """Separable linear interpolation of a coarse array onto `shape` (end points aligned)."""
    out = a.astype(np.float32)
    for ax, n in enumerate(shape):
        m = out.shape[ax]
        if m == n:
            continue
        x = np.linspace(0.0, m - 1.0, n)
        i0 = np.clip(np.floor(x).astype(np.int64), 0, m - 1)
        i1 = np.minimum(i0 + 1, m - 1)
        f = (x - i0).astype(np.float32)
        sh = [1] * out.ndim
        sh[ax] = n
        f = f.reshape(sh)
        out = np.take(out, i0, axis=ax) * (1.0 - f) + np.take(out, i1, axis=ax) * f
    return out


def gaussian_random_field(rng, shape, h: float, ell: float, std: float) -> np.ndarray:
    """White N(0,1) noise convolved with a Gaussian of standard deviation ell/2, so the
    covariance is proportional to exp(-r^2 / ell^2); normalised to `std`.  The field is
    drawn on a grid no finer than ell/4 and interpolated linearly onto `shape`."""
    from scipy.ndimage import gaussian_filter

    coarse_h = max(h, ell / 4.0)
    cshape = tuple(max(4, int(math.ceil((n - 1) * h / coarse_h)) + 1) for n in shape)
    white = rng.standard_normal(cshape, dtype=np.float32)
    f = gaussian_filter(white, sigma=(ell / 2.0) / coarse_h, mode="wrap")
    f = _upsample_linear(f, shape)
    f -= f.mean()
    s = float(f.std())
    return (f * (std / s if s > 0 else 0.0)).astype(np.float32)


def _layer_velocity(rng, depth_m: np.ndarray, nlayers: int, zmax: float, vtop: float,
                    vbot: float, jitter: float) -> np.ndarray:
    """Velocity of seeded horizontal layers evaluated at depths `depth_m`."""
    tops = np.sort(rng.uniform(0.05 * zmax, 0.95 * zmax, nlayers - 1))
    vel = np.linspace(vtop, vbot, nlayers) + rng.uniform(-jitter, jitter, nlayers)
    idx = np.searchsorted(tops, depth_m, side="right")
    return vel[idx].astype(np.float32)


@dataclass
class Workload:
    name: str
    ndim: int
    shape: tuple            # physical grid: (nz, nx) in 2-D, (nz, ny, nx) in 3-D
    h: float
    dt: float
    nt: int
    order: int
    f0: float
    src: np.ndarray         # int32 [nshots][3] (iz, iy, ix), iy = 0 in 2-D
    rec: np.ndarray         # int32 [nrec][3]  (shared by every shot)
    v: np.ndarray           # float32 velocity, physical grid
    v_obs: Optional[np.ndarray] = None  # model that produces the observed data
    nb: int = 20
    snap_dtype: str = "fp32"
    extra: dict = field(default_factory=dict)

    @property
    def nshots(self) -> int:
        return int(self.src.shape[0])

    @property
    def nrec(self) -> int:
        return int(self.rec.shape[0])

    def wavelets(self) -> np.ndarray:
        w = ricker(self.f0, self.dt, self.nt)
        return np.ascontiguousarray(np.broadcast_to(w, (self.nshots, self.nt)))

    def computed_points(self) -> int:
        n = 1
        for s in self.shape:
            n *= s + 2 * self.nb
        return n


def _surface_receivers_3d(ny, nx, iz, step):
    iy, ix = np.meshgrid(np.arange(0, ny, step), np.arange(0, nx, step), indexing="ij")
    r = np.stack([np.full(iy.size, iz), iy.ravel(), ix.ravel()], axis=1)
    return r.astype(np.int32)


def two_layer_2d(n: int = 201, nt: int = 500) -> Workload:
    """2-D two-layer model: 1500 m/s above row n//2, 2500 m/s from it down."""
    v = np.full((n, n), 1500.0, dtype=np.float32)
    v[n // 2:, :] = 2500.0
    src = np.array([[10, 0, n // 2]], dtype=np.int32)
    rec = np.stack([np.full(n, 5), np.zeros(n), np.arange(n)], axis=1).astype(np.int32)
    return Workload("two_layer_2d", 2, (n, n), 10.0, 1e-3, nt, 8, 15.0, src, rec, v)


def layered_3d(n: int = 256, nt: int = 2000, h: float = 10.0, dt: float = 0.8e-3,
               config_id: int = 2, snap_dtype: str = "bf16") -> Workload:
    """3-D layered model with smooth Gaussian random perturbations."""
    rng = rng_for(config_id)
    zmax = (n - 1) * h
    depth = np.arange(n, dtype=np.float64) * h
    vz = _layer_velocity(rng, depth, 8, zmax, 1500.0, 4500.0, 100.0)
    v = np.broadcast_to(vz[:, None, None], (n, n, n)).astype(np.float32)
    da = gaussian_random_field(rng, (n, n, n), h, 200.0, 0.05)
    db = gaussian_random_field(rng, (n, n, n), h, 200.0, 0.05)
    v_true = np.clip(v * (1.0 + da), 1500.0, 4500.0).astype(np.float32)
    v_obs = np.clip(v_true * (1.0 + db), 1500.0, 4500.0).astype(np.float32)
    step = 2 if n >= 64 else 1
    rec = _surface_receivers_3d(n, n, 5, step)
    src = np.array([[10, n // 2, n // 2]], dtype=np.int32)
    return Workload(f"layered_3d_{n}", 3, (n, n, n), h, dt, nt, 8, 15.0, src, rec, v_true,
                    v_obs, snap_dtype=snap_dtype)


def _fault_shift_2d(rng, nz, nx, nfaults):
    """Per-cell vertical throw (cells) from `nfaults` dipping normal faults."""
    zz, xx = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
    shift = np.zeros((nz, nx), dtype=np.float64)
    for _ in range(nfaults):
        x0 = rng.uniform(0.2, 0.8) * nx
        dip = math.radians(rng.uniform(30.0, 75.0))
        throw = rng.uniform(10.0, 40.0)
        hanging = xx > x0 + zz / math.tan(dip)
        shift += np.where(hanging, throw, 0.0)
    return shift


def faulted_2d(nz: int = 400, nx: int = 1024, nt: int = 3000, nshots: int = 64,
               config_id: int = 3) -> Workload:
    """2-D layered model with three dipping faults and a high-velocity salt ellipse."""
    rng = rng_for(config_id)
    h = 10.0
    shift = _fault_shift_2d(rng, nz, nx, 3)
    depth = (np.arange(nz)[:, None] - shift) * h
    v = _layer_velocity(rng, depth.ravel(), 6, (nz - 1) * h, 1500.0, 3500.0, 0.0)
    v = v.reshape(nz, nx)
    cx = rng.uniform(0.3, 0.7) * nx
    cz = rng.uniform(0.4, 0.7) * nz
    a = rng.uniform(60.0, 150.0) * nx / 1024.0
    b = rng.uniform(25.0, 60.0) * nz / 400.0
    zz, xx = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
    v[((xx - cx) / a) ** 2 + ((zz - cz) / b) ** 2 <= 1.0] = 4500.0
    v = v.astype(np.float32)
    db = gaussian_random_field(rng, (nz, nx), h, 200.0, 0.05)
    v_obs = np.clip(v * (1.0 + db), 1500.0, 4500.0).astype(np.float32)
    spacing = nx / nshots
    six = (spacing / 2 + spacing * np.arange(nshots)).astype(np.int64)
    src = np.stack([np.full(nshots, 10), np.zeros(nshots), six], axis=1).astype(np.int32)
    rec = np.stack([np.full(nx, 5), np.zeros(nx), np.arange(nx)], axis=1).astype(np.int32)
    return Workload(f"faulted_2d_{nz}x{nx}x{nshots}", 2, (nz, nx), h, 1e-3, nt, 8, 20.0,
                    src, rec, v, v_obs, snap_dtype="bf16")


def salt_3d(n: int = 512, nt: int = 4000, config_id: int = 5,
            snap_dtype: str = "fp16") -> Workload:
    """3-D layered model with three dipping fault planes and a salt ellipsoid; `n` < 512
    gives a twin with the same physical size (h = 12.5 m * 512 / n, dt scaled alike)."""
    rng = rng_for(config_id)
    h = 12.5 * 512.0 / n
    dt = 0.6e-3 * 512.0 / n
    nt = int(round(nt * n / 512.0))
    zz, yy, xx = np.meshgrid(np.arange(n, dtype=np.float32), np.arange(n, dtype=np.float32),
                             np.arange(n, dtype=np.float32), indexing="ij")
    shift = np.zeros((n, n, n), dtype=np.float32)
    for _ in range(3):
        x0, y0 = rng.uniform(0.2, 0.8, 2) * n
        strike = rng.uniform(0.0, 2.0 * math.pi)
        dip = math.radians(rng.uniform(30.0, 75.0))
        throw = rng.uniform(10.0, 40.0) * n / 512.0
        side = (xx - x0) * math.cos(strike) + (yy - y0) * math.sin(strike)
        shift += np.where(side > zz / math.tan(dip), np.float32(throw), np.float32(0.0))
    depth = (zz - shift) * h
    del shift, side
    v = _layer_velocity(rng, depth.ravel(), 10, (n - 1) * h, 1500.0, 4500.0, 0.0)
    v = v.reshape(n, n, n)
    del depth
    c = rng.uniform([0.4, 0.3, 0.3], [0.7, 0.7, 0.7]) * n
    ax = rng.uniform([25.0, 60.0, 60.0], [60.0, 150.0, 150.0]) * n / 512.0
    inside = (((zz - c[0]) / ax[0]) ** 2 + ((yy - c[1]) / ax[1]) ** 2
              + ((xx - c[2]) / ax[2]) ** 2) <= 1.0
    v[inside] = 4500.0
    del zz, yy, xx, inside
    db = gaussian_random_field(rng, (n, n, n), h, 200.0, 0.05)
    v_obs = np.clip(v * (1.0 + db), 1500.0, 4500.0).astype(np.float32)
    step = 2 if n >= 64 else 1
    rec = _surface_receivers_3d(n, n, 5, step)
    src = np.array([[10, n // 2, n // 2]], dtype=np.int32)
    # the peak frequency scales with the grid so a twin keeps the points per wavelength
    return Workload(f"salt_3d_{n}", 3, (n, n, n), h, dt, nt, 16, 15.0 * n / 512.0,
                    src, rec, v, v_obs, snap_dtype=snap_dtype)


def smooth_random(rng, shape, h: float, ell: float = 300.0) -> np.ndarray:
    """Smooth random velocity: a Gaussian random field mapped monotonically onto
    1500..4500 m/s through its rank-free affine rescaling."""
    f = gaussian_random_field(rng, shape, h, ell, 1.0)
    lo, hi = float(f.min()), float(f.max())
    if hi - lo < 1e-12:
        return np.full(shape, 3000.0, dtype=np.float32)
    return (1500.0 + 3000.0 * (f - lo) / (hi - lo)).astype(np.float32)


def serving_requests(n: int, dt_for, seed: int = 4, size2d=(128, 1024), size3d=(64, 192),
                     nt_range=(500, 3000), frac_grad: float = 0.5, frac_2d: float = 0.75,
                     h: float = 10.0):
    """Request mix of the serving workload: 2-D grids with sides ~U{size2d}, 3-D grids
    with sides ~U{size3d}, nt ~U{nt_range}, forward or gradient, smooth random velocity
    (Gaussian random field, correlation length 300 m, mapped onto 1500..4500 m/s),
    source at the surface centre (row 2), receivers on every cell of row 2, 8th order,
    BF16 checkpoints, 15 Hz Ricker.  dt_for(ndim, h) gives the time step (the caller's
    rule, e.g. 0.8 of the stability limit).  The observed model of a gradient request is
    its velocity times (1 + 5 % random field).  Arrival times are left at 0; the caller
    draws them."""
    rng = rng_for(4, 1000 + seed)
    reqs = []
    for i in range(n):
        is2d = rng.random() < frac_2d
        kind = "gradient" if rng.random() < frac_grad else "forward"
        nt = int(rng.integers(nt_range[0], nt_range[1] + 1))
        if is2d:
            nz, nx = (int(x) for x in rng.integers(size2d[0], size2d[1] + 1, 2))
            shape = (nz, nx)
            ndim = 2
        else:
            shape = tuple(int(x) for x in rng.integers(size3d[0], size3d[1] + 1, 3))
            ndim = 3
        v = smooth_random(rng, shape, h, ell=300.0)
        dt = float(dt_for(ndim, h))
        if ndim == 2:
            src = [2, 0, shape[1] // 2]
            rec = np.stack([np.full(shape[1], 2), np.zeros(shape[1]), np.arange(shape[1])], 1)
        else:
            src = [2, shape[1] // 2, shape[2] // 2]
            yy, xx = np.meshgrid(np.arange(shape[1]), np.arange(shape[2]), indexing="ij")
            rec = np.stack([np.full(yy.size, 2), yy.ravel(), xx.ravel()], 1)
        r = {"kind": kind, "v": v, "h": h, "dt": dt, "nt": nt, "order": 8, "snap_dtype": "bf16",
             "src": src, "rec": rec.astype(np.int32), "wavelet": ricker(15.0, dt, nt),
             "arrival": 0.0}
        if kind == "gradient":
            r["v_obs"] = (v * (1.0 + gaussian_random_field(rng, shape, h, 200.0, 0.05))).astype(np.float32)
        reqs.append(r)
    return reqs


def random_small(rng, ndim: int, shape, h: float = 10.0, nt: int = 60, order: int = 8,
                 nb: int = 6, nrec: int = 7, f0: float = 20.0) -> Workload:
    """Small random case for parity tests: smooth random model, random source and
    receiver nodes anywhere in the physical grid (tile edges included)."""
    shape = tuple(int(s) for s in shape)
    v = smooth_random(rng, shape, h, ell=8 * h)
    if ndim == 2:
        nz, nx = shape
        src = np.array([[rng.integers(nz), 0, rng.integers(nx)]], dtype=np.int32)
        rec = np.stack([rng.integers(0, nz, nrec), np.zeros(nrec, dtype=np.int64),
                        rng.integers(0, nx, nrec)], axis=1).astype(np.int32)
    else:
        nz, ny, nx = shape
        src = np.array([[rng.integers(nz), rng.integers(ny), rng.integers(nx)]],
                       dtype=np.int32)
        rec = np.stack([rng.integers(0, nz, nrec), rng.integers(0, ny, nrec),
                        rng.integers(0, nx, nrec)], axis=1).astype(np.int32)
    vmax = 4500.0
    M = order // 2
    # half of the stability limit of the 2M-order leapfrog for this grid (host check)
    dt = 0.4 * h / vmax
    return Workload(f"random_{ndim}d_{'x'.join(map(str, shape))}", ndim, shape, h, dt, nt,
                    order, f0 if f0 else 20.0, src, rec, v, nb=nb,
                    extra={"M": M})
