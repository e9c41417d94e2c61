"""FP64 CPU oracle for the FWI hot path (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
import this package.  The product path (``paper_1912_08063_gb300``) never does: it has
no CPU fallback.  The oracle shares no code with the CUDA library; the two meet only at
the seeded synthetic inputs (``paper_1912_08063_gb300.synth``), which carry none of the
method's arithmetic.

The arithmetic lives in ``fwi_oracle.c`` (plain C loops in double precision).  This
module compiles it on first use with gcc and wraps it with ctypes; the wrappers only
convert arrays.  See the C file's header for the equations each function follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fwi_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc -O2 -fopenmp, no fast-math)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _configure(ctypes.CDLL(build()))
    return _lib


def compile_source(text: str, out_path: str) -> str:
    """Compiles C source text with the oracle's flags (used by the tests that plant a
    mistake in a copy of the oracle and check that a pin catches it)."""
    src = out_path + ".c"
    with open(src, "w") as f:
        f.write(text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
                    "-ffp-contract=off", src, "-o", out_path, "-lm"], check=True)
    return out_path


class use_library:
    """Context manager: route every oracle call to the library at `path`."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        _load()
        self.saved = _lib
        _lib = _configure(ctypes.CDLL(self.path))
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def _configure(lib):
    """Declares the argument and result types of every oracle function on `lib`."""
    P = ctypes.c_void_p
    i64p = ctypes.POINTER(ctypes.c_int64)
    d = ctypes.c_double
    i = ctypes.c_int
    lib.oracle_fd_coeffs.argtypes = [i, P]
    lib.oracle_fd_coeffs.restype = i
    lib.oracle_cfl_number.argtypes = [i, i, P, d, d]
    lib.oracle_cfl_number.restype = d
    lib.oracle_laplacian.argtypes = [i, i64p, P, i, P, P]
    lib.oracle_laplacian.restype = i
    common = [i, i64p, P, P, d, i, i, i, d, d]
    lib.oracle_forward.argtypes = common + [i, P, P, P, i, P, P, P, P]
    lib.oracle_forward.restype = i
    lib.oracle_misfit.argtypes = [P, P, ctypes.c_int64]
    lib.oracle_misfit.restype = d
    lib.oracle_gradient.argtypes = common + [i, P, P, P, i, P, P, P, P, P, P, P, i]
    lib.oracle_gradient.restype = i
    lib.oracle_source_adjoint.argtypes = common + [i, P, P, i, P, P, P, P]
    lib.oracle_source_adjoint.restype = i
    lib.oracle_point_taps.argtypes = [i, i64p, i, P, P, P]
    lib.oracle_point_taps.restype = i
    lib.oracle_model_fields.argtypes = [i, i64p, P, P, d, i, i, d, d, i64p, P, P, P]
    lib.oracle_model_fields.restype = i
    f = ctypes.c_float
    u16 = ctypes.c_uint16
    lib.oracle_snap_scale.argtypes = [f, i]
    lib.oracle_snap_scale.restype = f
    lib.oracle_f32_to_bf16.argtypes = [f]
    lib.oracle_f32_to_bf16.restype = u16
    lib.oracle_f32_to_f16.argtypes = [f]
    lib.oracle_f32_to_f16.restype = u16
    lib.oracle_bf16_to_f32.argtypes = [u16]
    lib.oracle_bf16_to_f32.restype = f
    lib.oracle_f16_to_f32.argtypes = [u16]
    lib.oracle_f16_to_f32.restype = f
    lib.oracle_snap_encode.argtypes = [P, P, ctypes.c_int64, i, P, P]
    lib.oracle_snap_encode.restype = None
    lib.oracle_snap_decode.argtypes = [P, P, ctypes.c_int64, i, P, P]
    lib.oracle_snap_decode.restype = None
    return lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _shape3(ndim, shape):
    shape = tuple(int(s) for s in shape)
    if ndim == 2:
        if len(shape) == 2:
            shape = (shape[0], 1, shape[1])
    if len(shape) != 3:
        raise ValueError("shape must be (nz, nx) in 2-D or (nz, ny, nx) in 3-D")
    return (ctypes.c_int64 * 3)(*shape), shape


def _h3(ndim, h):
    h = [float(x) for x in np.atleast_1d(h)]
    if len(h) == 1:
        h = h * 3
    if ndim == 2 and len(h) == 2:
        h = [h[0], 1.0, h[1]]
    return _f64(h)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def order_to_radius(order: int) -> int:
    """Stencil order 2M -> radius M (8th order: 4, 16th order: 8)."""
    if order % 2 or not 2 <= order <= 16:
        raise ValueError("order must be even, 2..16")
    return order // 2


def fd_coeffs(M: int) -> np.ndarray:
    c = np.zeros(M + 1)
    _check(_load().oracle_fd_coeffs(M, _ptr(c)), "fd_coeffs")
    return c


def cfl_number(ndim, M, h, vmax, dt) -> float:
    return _load().oracle_cfl_number(ndim, M, _ptr(_h3(ndim, h)), float(vmax), float(dt))


def laplacian(u, h, M):
    """L u on a grid with zero outside (2-D arrays are (nz, nx), 3-D (nz, ny, nx))."""
    u = _f64(u)
    ndim = u.ndim
    shp, _ = _shape3(ndim, u.shape)
    out = np.empty_like(u)
    _check(_load().oracle_laplacian(ndim, shp, _ptr(_h3(ndim, h)), M, _ptr(u), _ptr(out)),
           "laplacian")
    return out


def point_taps(shape, pos, nb=20):
    """(cell indices on the computed grid, weights) of the Kaiser-windowed sinc point at
    `pos` ((z, x) or (z, y, x) physical-grid index units) for a grid of physical
    `shape`."""
    ndim = len(shape)
    shp, _ = _shape3(ndim, shape)
    p = _f64(pos)
    if ndim == 2:
        p = np.array([p[0], 0.0, p[1]])
    idx = np.zeros(512, dtype=np.int64)
    w = np.zeros(512)
    T = _load().oracle_point_taps(ndim, shp, int(nb), _ptr(p), _ptr(idx), _ptr(w))
    if T < 0:
        raise ValueError("point outside the grid")
    return idx[:T], w[:T]


class Problem:
    """Arguments shared by every oracle call (physical grid, numerics, acquisition)."""

    def __init__(self, v, h, dt, nt, order=8, nb=20, r0=1e-3, vref=0.0,
                 src=None, rec=None, wavelet=None, src_pos=None, rec_pos=None):
        """src/rec: grid nodes (z, y, x); src_pos/rec_pos, when given, are fractional
        positions in the same index units (Kaiser-windowed sinc points) and replace
        the nodes."""
        self.v = _f64(v)
        self.ndim = self.v.ndim
        self.shape_c, self.shape = _shape3(self.ndim, self.v.shape)
        self.h = _h3(self.ndim, h)
        self.dt = float(dt)
        self.nt = int(nt)
        self.M = order_to_radius(order)
        self.nb = int(nb)
        self.r0 = float(r0)
        self.vref = float(vref)
        if src is None:
            src = np.rint(np.asarray(src_pos, dtype=np.float64))
        if rec is None:
            rec = np.rint(np.asarray(rec_pos, dtype=np.float64))
        self.src = _i32(src).reshape(-1, 3)
        self.nshots = self.src.shape[0]
        rec = _i32(rec)
        if rec.ndim == 2:
            rec = np.broadcast_to(rec, (self.nshots,) + rec.shape)
        self.rec = _i32(rec).reshape(self.nshots, -1, 3)
        self.nrec = self.rec.shape[1]
        self.src_pos = None if src_pos is None else _f64(src_pos).reshape(self.nshots, 3)
        if rec_pos is not None:
            rp = _f64(rec_pos)
            if rp.ndim == 2:
                rp = np.broadcast_to(rp, (self.nshots,) + rp.shape)
            rec_pos = _f64(rp).reshape(self.nshots, self.nrec, 3)
        self.rec_pos = rec_pos
        w = _f64(wavelet)
        if w.ndim == 1:
            w = np.broadcast_to(w, (self.nshots, w.shape[0]))
        self.wavelet = _f64(w).reshape(self.nshots, self.nt)

    def _common(self, v=None):
        v = self.v if v is None else _f64(v)
        return [self.ndim, self.shape_c, _ptr(self.h), _ptr(v), self.dt, self.nt, self.M,
                self.nb, self.r0, self.vref]

    def computed_shape(self):
        nb = self.nb
        nz, ny, nx = self.shape
        if self.ndim == 2:
            return (nz + 2 * nb, nx + 2 * nb)
        return (nz + 2 * nb, ny + 2 * nb, nx + 2 * nb)

    def forward(self, v=None, wavelet=None, final=False):
        """Traces [nshots][nt][nrec]; with final=True also (u^nt, u^{nt-1}) per shot."""
        w = self.wavelet if wavelet is None else _f64(wavelet).reshape(self.nshots, self.nt)
        tr = np.zeros((self.nshots, self.nt, self.nrec))
        cs = self.computed_shape()
        fin = np.zeros((self.nshots, 2) + cs) if final else None
        rc = _load().oracle_forward(*self._common(v), self.nshots, _ptr(self.src),
                                    _ptr(self.src_pos), _ptr(w), self.nrec, _ptr(self.rec),
                                    _ptr(self.rec_pos), _ptr(tr), _ptr(fin))
        _check(rc, "forward")
        return (tr, fin) if final else tr

    def gradient(self, dobs=None, v=None, adjsrc=None, seg=None, want_gW=False):
        """(misfit, d misfit / d v on the physical grid[, d misfit / d W computed grid])."""
        seg = seg or max(1, int(round(np.sqrt(self.nt))))
        grad = np.zeros(self.shape if self.ndim == 3 else (self.shape[0], self.shape[2]))
        gW = np.zeros(self.computed_shape()) if want_gW else None
        phi = ctypes.c_double(0.0)
        dobs_a = None if dobs is None else _f64(dobs)
        adj_a = None if adjsrc is None else _f64(adjsrc)
        if dobs_a is None and adj_a is None:
            raise ValueError("need dobs or adjsrc")
        rc = _load().oracle_gradient(*self._common(v), self.nshots, _ptr(self.src),
                                     _ptr(self.src_pos), _ptr(self.wavelet), self.nrec,
                                     _ptr(self.rec), _ptr(self.rec_pos),
                                     _ptr(dobs_a), _ptr(adj_a), ctypes.byref(phi),
                                     _ptr(grad), _ptr(gW), int(seg))
        _check(rc, "gradient")
        if want_gW:
            return phi.value, grad, gW
        return phi.value, grad

    def source_adjoint(self, y):
        y = _f64(y).reshape(self.nshots, self.nt, self.nrec)
        x = np.zeros((self.nshots, self.nt))
        rc = _load().oracle_source_adjoint(*self._common(), self.nshots, _ptr(self.src),
                                           _ptr(self.src_pos), self.nrec, _ptr(self.rec),
                                           _ptr(self.rec_pos), _ptr(y), _ptr(x))
        _check(rc, "source_adjoint")
        return x

    def fields(self):
        """(W, a+, a-) on the computed grid."""
        cs = self.computed_shape()
        W, ap, am = np.zeros(cs), np.zeros(cs), np.zeros(cs)
        nc = (ctypes.c_int64 * 3)()
        rc = _load().oracle_model_fields(self.ndim, self.shape_c, _ptr(self.h), _ptr(self.v),
                                         self.dt, self.M, self.nb, self.r0, self.vref, nc,
                                         _ptr(W), _ptr(ap), _ptr(am))
        _check(rc, "model_fields")
        return W, ap, am


def misfit(dmod, dobs) -> float:
    a, b = _f64(dmod), _f64(dobs)
    return _load().oracle_misfit(_ptr(a), _ptr(b), a.size)


SNAP = {"fp32": 0, "bf16": 1, "fp16": 2}


def snap_scale(maxabs: float, dtype: str) -> float:
    return _load().oracle_snap_scale(float(maxabs), SNAP[dtype])


def snap_encode(a, b, dtype: str):
    """(codes uint16 [2][n], scales float32 [2]) of the checkpoint pair (a, b): the
    components a and a - b, each with its own power-of-two scale."""
    a = np.ascontiguousarray(a, dtype=np.float32).ravel()
    b = np.ascontiguousarray(b, dtype=np.float32).ravel()
    code = np.zeros((2, a.size), dtype=np.uint16)
    sc = np.zeros(2, dtype=np.float32)
    _load().oracle_snap_encode(_ptr(a), _ptr(b), a.size, SNAP[dtype], _ptr(code), _ptr(sc))
    return code, sc


def snap_decode(code, scales, dtype: str):
    code = np.ascontiguousarray(code, dtype=np.uint16).reshape(2, -1)
    sc = np.ascontiguousarray(scales, dtype=np.float32).reshape(2)
    n = code.shape[1]
    a = np.zeros(n, dtype=np.float32)
    b = np.zeros(n, dtype=np.float32)
    _load().oracle_snap_decode(_ptr(code), _ptr(sc), n, SNAP[dtype], _ptr(a), _ptr(b))
    return a, b


def f32_to_bf16(x) -> np.ndarray:
    f = _load().oracle_f32_to_bf16
    return np.array([f(float(v)) for v in np.asarray(x, dtype=np.float32).ravel()],
                    dtype=np.uint16)


def f32_to_f16(x) -> np.ndarray:
    f = _load().oracle_f32_to_f16
    return np.array([f(float(v)) for v in np.asarray(x, dtype=np.float32).ravel()],
                    dtype=np.uint16)
