"""Python binding of libfwi (include/fwi.h): argument marshalling only.

Every function of the C ABI is exposed under the same name; ``FwiModel`` wraps a model
handle for torch tensors and numpy arrays.  Every step of the hot path runs in the CUDA
library.  There is no CPU fallback: importing a function that needs the library raises
when ``libfwi.so`` cannot be built or loaded.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

import numpy as np

from . import build as _build

FWI_OK = 0
FWI_ERR_ARG = -1
FWI_ERR_CFL = -2
FWI_ERR_OOM = -3
FWI_ERR_CUDA = -4
FWI_ERR_UNSTABLE = -5
FWI_ERR_TIMEOUT = -6
SNAP_DTYPES = {"fp32": 0, "bf16": 1, "fp16": 2}
ERR_NAMES = {0: "FWI_OK", -1: "FWI_ERR_ARG", -2: "FWI_ERR_CFL", -3: "FWI_ERR_OOM",
             -4: "FWI_ERR_CUDA", -5: "FWI_ERR_UNSTABLE", -6: "FWI_ERR_TIMEOUT"}

c_i32, c_i64, c_f32, c_f64, c_vp = (ctypes.c_int32, ctypes.c_int64, ctypes.c_float,
                                    ctypes.c_double, ctypes.c_void_p)


class fwi_opts(ctypes.Structure):
    _fields_ = [("order", c_i32), ("nb", c_i32), ("snap_dtype", c_i32), ("fold_every", c_i32),
                ("snap_budget_bytes", c_i64), ("sponge_r0", c_f32), ("sponge_vref", c_f32),
                ("timing", c_i32), ("temporal_blocking", c_i32)]


class fwi_acq(ctypes.Structure):
    _fields_ = [("nshots", c_i32), ("nrec", c_i32), ("src", c_vp), ("rec", c_vp),
                ("src_pos", c_vp), ("rec_pos", c_vp)]


class fwi_info(ctypes.Structure):
    _fields_ = [("ndim", c_i32), ("order", c_i32), ("nb", c_i32), ("nt", c_i32),
                ("shape", c_i64 * 3), ("computed", c_i64 * 3), ("pitch_x", c_i64),
                ("points", c_i64), ("device_bytes", c_i64), ("snap_slots", c_i32),
                ("shots_capacity", c_i32), ("last_forward_steps", c_i64),
                ("last_adjoint_steps", c_i64), ("last_snap_stores", c_i64),
                ("last_snap_restores", c_i64), ("sponge_eta_max", c_f32 * 3), ("cfl", c_f32),
                ("kernel_launches", c_i64), ("fwd_step_launches", c_i64),
                ("adj_step_launches", c_i64), ("fwd_step_ms", c_f64), ("adj_step_ms", c_f64),
                ("store_step_launches", c_i64), ("store_step_ms", c_f64),
                ("step_ctas", c_i32 * 3), ("reserved2", c_i32)]


class fwi_request(ctypes.Structure):
    _fields_ = [("kind", c_i32), ("ndim", c_i32), ("shape", c_i64 * 3), ("spacing", c_f32 * 3),
                ("dt", c_f32), ("nt", c_i32), ("order", c_i32), ("snap_dtype", c_i32),
                ("nrec", c_i32), ("src", c_i32 * 3), ("reserved", c_i32), ("vp", c_vp),
                ("wavelet", c_vp), ("rec", c_vp), ("d_obs", c_vp), ("traces_out", c_vp),
                ("grad_out", c_vp), ("arrival", c_f64)]


class fwi_result(ctypes.Structure):
    _fields_ = [("status", c_i32), ("shared_launch", c_i32), ("misfit", c_f64), ("t_admit", c_f64),
                ("t_start", c_f64), ("t_done", c_f64), ("device_bytes", c_i64),
                ("reserved_bytes", c_i64)]


class fwi_serve_opts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", c_i64), ("max_active", c_i32), ("steps_per_turn", c_i32),
                ("snap_slots", c_i32), ("nb", c_i32), ("no_shared_launch", c_i32)]


class FwiError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None
_lock = threading.Lock()


def lib():
    """The loaded libfwi (built in-tree on first use)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            P = c_vp
            sig = {
                "fwi_create_model": ([P, c_i32, P, P, P, c_f32, c_i32, P, P], c_i32),
                "fwi_update_velocity": ([P, P, P], c_i32),
                "fwi_forward": ([P, P, P, P, P, P], c_i32),
                "fwi_adjoint_gradient": ([P, P, P, P, P, P, P, P], c_i32),
                "fwi_source_adjoint": ([P, P, P, P, P], c_i32),
                "fwi_misfit": ([P, P, c_i64, P, P], c_i32),
                "fwi_misfit_noalloc": ([P, P, c_i64, P, P], c_i32),
                "fwi_snapshot_encode": ([P, P, c_i64, c_i32, P, P, P], c_i32),
                "fwi_snapshot_decode": ([P, P, c_i64, c_i32, P, P, P], c_i32),
                "fwi_revolve_schedule": ([c_i32, c_i32, P, c_i64, P, P], c_i32),
                "fwi_checkpoint_plan": ([c_i32, c_i64, P, P, P], c_i32),
                "fwi_fd_coeffs": ([c_i32, P], c_i32),
                "fwi_cfl_number": ([c_i32, c_i32, P, c_f32, c_f32], c_f64),
                "fwi_model_info": ([P, P], c_i32),
                "fwi_serve": ([P, c_i32, P, P], c_i32),
                "fwi_sync_status": ([P], c_i32),
                "fwi_selftest_wait": ([P, c_i32, P], c_i32),
                "fwi_destroy": ([P], None),
                "fwi_last_error": ([], ctypes.c_char_p),
            }
            for name, (args, res) in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def _check(rc: int):
    if rc != FWI_OK:
        raise FwiError(rc, lib().fwi_last_error().decode())


def _ptr(x) -> Optional[int]:
    """Address of a torch tensor or numpy array (None passes NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("arrays must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr()
    raise TypeError(f"unsupported buffer type {type(x)}")


def _stream(stream) -> Optional[int]:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    return int(getattr(stream, "cuda_stream", stream))


# ---------------------------------------------------------------- C ABI, same names

def fwi_create_model(ndim, shape, spacing, vp, dt, nt, opts: Optional[fwi_opts] = None,
                     stream=None) -> int:
    h = c_vp()
    shp = (c_i64 * 3)(*[int(s) for s in shape])
    sp = (c_f32 * 3)(*[float(s) for s in spacing])
    _check(lib().fwi_create_model(ctypes.byref(h), int(ndim), shp, sp, _ptr(vp), float(dt),
                                  int(nt), ctypes.byref(opts) if opts is not None else None,
                                  _stream(stream)))
    return h.value


def fwi_update_velocity(model, vp, stream=None):
    _check(lib().fwi_update_velocity(model, _ptr(vp), _stream(stream)))


def fwi_forward(model, acq: fwi_acq, wavelets, traces, final_state=None, stream=None):
    _check(lib().fwi_forward(model, ctypes.byref(acq), _ptr(wavelets), _ptr(traces),
                             _ptr(final_state), _stream(stream)))


def fwi_adjoint_gradient(model, acq: fwi_acq, wavelets, d_obs, misfit, grad, grad64=None,
                         stream=None):
    _check(lib().fwi_adjoint_gradient(model, ctypes.byref(acq), _ptr(wavelets), _ptr(d_obs),
                                      _ptr(misfit), _ptr(grad), _ptr(grad64), _stream(stream)))


def fwi_source_adjoint(model, acq: fwi_acq, y, x, stream=None):
    _check(lib().fwi_source_adjoint(model, ctypes.byref(acq), _ptr(y), _ptr(x),
                                    _stream(stream)))


def fwi_misfit(d_mod, d_obs, n, misfit_dev, stream=None):
    _check(lib().fwi_misfit(_ptr(d_mod), _ptr(d_obs), int(n), _ptr(misfit_dev),
                            _stream(stream)))


def fwi_misfit_noalloc(d_mod, d_obs, n, misfit_dev, stream=None):
    _check(lib().fwi_misfit_noalloc(_ptr(d_mod), _ptr(d_obs), int(n), _ptr(misfit_dev),
                                    _stream(stream)))


def fwi_snapshot_encode(a, b, n, dtype, code, scale, stream=None):
    _check(lib().fwi_snapshot_encode(_ptr(a), _ptr(b), int(n), int(dtype), _ptr(code),
                                     _ptr(scale), _stream(stream)))


def fwi_snapshot_decode(code, scale, n, dtype, a, b, stream=None):
    _check(lib().fwi_snapshot_decode(_ptr(code), _ptr(scale), int(n), int(dtype), _ptr(a),
                                     _ptr(b), _stream(stream)))


def fwi_revolve_schedule(nsteps: int, nslots: int):
    """(actions int32 [n][2], forward step count) of the binomial checkpoint schedule."""
    na, nf = c_i64(), c_i64()
    _check(lib().fwi_revolve_schedule(int(nsteps), int(nslots), None, 0, ctypes.byref(na),
                                      ctypes.byref(nf)))
    out = np.zeros((na.value, 2), dtype=np.int32)
    _check(lib().fwi_revolve_schedule(int(nsteps), int(nslots), out.ctypes.data, na.value,
                                      ctypes.byref(na), ctypes.byref(nf)))
    return out, nf.value


def fwi_checkpoint_plan(nsteps: int, half_slots: int):
    """(slots, pair slots, forward steps) of the checkpoint plan a gradient call makes for
    nsteps steps from a budget of half_slots field-sized units."""
    ns, npair, nf = c_i32(), c_i32(), c_i64()
    _check(lib().fwi_checkpoint_plan(int(nsteps), int(half_slots), ctypes.byref(ns),
                                     ctypes.byref(npair), ctypes.byref(nf)))
    return ns.value, npair.value, nf.value


def fwi_fd_coeffs(order: int) -> np.ndarray:
    c = np.zeros(order // 2 + 1)
    _check(lib().fwi_fd_coeffs(int(order), c.ctypes.data))
    return c


def fwi_cfl_number(ndim, order, spacing, vmax, dt) -> float:
    sp = (c_f32 * 3)(*[float(s) for s in spacing])
    return lib().fwi_cfl_number(int(ndim), int(order), sp, float(vmax), float(dt))


def fwi_model_info(model) -> dict:
    info = fwi_info()
    _check(lib().fwi_model_info(model, ctypes.byref(info)))
    out = {}
    for name, _ in fwi_info._fields_:
        v = getattr(info, name)
        out[name] = list(v) if hasattr(v, "__len__") else v
    return out


def fwi_serve(requests, budget_bytes=0, max_active=16, steps_per_turn=8, snap_slots=64, nb=20,
              shared_launch=True):
    """Runs a request stream through the serving loop.  `requests` is a list of dicts with
    keys kind ('forward'/'gradient'), v (float32 physical grid), h, dt, nt, order,
    snap_dtype, src (3 ints), rec (int32 [nrec][3]), wavelet (float32 [nt]), d_obs
    (float32 [nt][nrec], gradients) and arrival (s).  Returns (results as dicts, outputs):
    outputs[i] is the traces [nt][nrec] of a forward request or the gradient of a
    gradient request."""
    n = len(requests)
    arr = (fwi_request * n)()
    keep, outs = [], []
    for i, r in enumerate(requests):
        v = np.ascontiguousarray(r["v"], dtype=np.float32)
        ndim = v.ndim
        shape = v.shape if ndim == 3 else (v.shape[0], 1, v.shape[1])
        h = float(r["h"])
        wav = np.ascontiguousarray(r["wavelet"], dtype=np.float32)
        rec = np.ascontiguousarray(r["rec"], dtype=np.int32).reshape(-1, 3)
        nrec = rec.shape[0]
        grad = r["kind"] == "gradient"
        if grad:
            dobs = np.ascontiguousarray(r["d_obs"], dtype=np.float32)
            out = np.zeros(v.shape, dtype=np.float32)
        else:
            dobs = None
            out = np.zeros((int(r["nt"]), nrec), dtype=np.float32)
        keep += [v, wav, rec, dobs]
        outs.append(out)
        q = arr[i]
        q.kind = 1 if grad else 0
        q.ndim = ndim
        q.shape = (c_i64 * 3)(*shape)
        q.spacing = (c_f32 * 3)(h, h if ndim == 3 else 1.0, h)
        q.dt = float(r["dt"])
        q.nt = int(r["nt"])
        q.order = int(r.get("order", 8))
        q.snap_dtype = SNAP_DTYPES[r.get("snap_dtype", "bf16")]
        q.nrec = nrec
        q.src = (c_i32 * 3)(*[int(x) for x in r["src"]])
        q.vp = v.ctypes.data
        q.wavelet = wav.ctypes.data
        q.rec = rec.ctypes.data
        q.d_obs = dobs.ctypes.data if grad else None
        q.traces_out = None if grad else out.ctypes.data
        q.grad_out = out.ctypes.data if grad else None
        q.arrival = float(r.get("arrival", 0.0))
    res = (fwi_result * n)()
    opts = fwi_serve_opts(int(budget_bytes), int(max_active), int(steps_per_turn),
                          int(snap_slots), int(nb), 0 if shared_launch else 1)
    _check(lib().fwi_serve(arr, n, ctypes.byref(opts), res))
    results = [{k: getattr(x, k) for k, _ in fwi_result._fields_} for x in res]
    return results, outs


def fwi_sync_status(model):
    _check(lib().fwi_sync_status(model))


def fwi_selftest_wait(model, polls, stream=None):
    _check(lib().fwi_selftest_wait(model, int(polls), _stream(stream)))


def fwi_destroy(model):
    lib().fwi_destroy(model)


def fwi_last_error() -> str:
    return lib().fwi_last_error().decode()


# ---------------------------------------------------------------- convenience wrapper

class Acquisition:
    """Host-side source/receiver geometry kept alive for the duration of calls: grid nodes
    (src, rec as (z, y, x) integers) or off-grid positions (src_pos, rec_pos as
    fractional (z, y, x) index coordinates, Kaiser-windowed sinc points); a position
    array replaces the corresponding node array."""

    def __init__(self, src=None, rec=None, src_pos=None, rec_pos=None):
        if src is None:
            src = np.rint(np.asarray(src_pos, dtype=np.float64))
        if rec is None:
            rec = np.rint(np.asarray(rec_pos, dtype=np.float64))
        self.src = np.ascontiguousarray(np.asarray(src, dtype=np.int32).reshape(-1, 3))
        ns = self.src.shape[0]
        rec = np.asarray(rec, dtype=np.int32)
        if rec.ndim == 2:
            rec = np.broadcast_to(rec, (ns,) + rec.shape)
        self.rec = np.ascontiguousarray(rec.reshape(ns, -1, 3))
        nr = self.rec.shape[1]
        self.src_pos = None if src_pos is None else np.ascontiguousarray(
            np.asarray(src_pos, dtype=np.float64).reshape(ns, 3))
        self.rec_pos = None
        if rec_pos is not None:
            rp = np.asarray(rec_pos, dtype=np.float64)
            if rp.ndim == 2:
                rp = np.broadcast_to(rp, (ns,) + rp.shape)
            self.rec_pos = np.ascontiguousarray(rp.reshape(ns, nr, 3))
        self.c = fwi_acq(ns, nr, self.src.ctypes.data, self.rec.ctypes.data,
                         None if self.src_pos is None else self.src_pos.ctypes.data,
                         None if self.rec_pos is None else self.rec_pos.ctypes.data)

    @property
    def nshots(self):
        return self.src.shape[0]

    @property
    def nrec(self):
        return self.rec.shape[1]


class FwiModel:
    """A velocity model on the device with its numerics; methods mirror the C ABI."""

    def __init__(self, v, spacing, dt, nt, order=8, nb=20, snap_dtype="fp32",
                 snap_budget_bytes=0, sponge_r0=1e-3, sponge_vref=0.0, fold_every=256,
                 timing=False, stream=None, temporal_blocking=False):
        import torch
        if isinstance(v, np.ndarray):
            v = torch.from_numpy(np.ascontiguousarray(v, dtype=np.float32))
        v = v.contiguous()
        if v.dtype != torch.float32:
            v = v.float()
        self.ndim = v.dim()
        self.shape = tuple(v.shape) if self.ndim == 3 else (v.shape[0], 1, v.shape[1])
        sp = list(np.atleast_1d(np.asarray(spacing, dtype=np.float64)))
        if len(sp) == 1:
            sp = sp * 3
        elif len(sp) == 2:
            sp = [sp[0], 1.0, sp[1]]
        self.spacing = sp
        self.dt, self.nt, self.order = float(dt), int(nt), int(order)
        self.opts = fwi_opts(int(order), int(nb) if nb else -1, SNAP_DTYPES[snap_dtype],
                             int(fold_every), int(snap_budget_bytes), float(sponge_r0),
                             float(sponge_vref), int(bool(timing)),
                             int(temporal_blocking))
        self.handle = fwi_create_model(self.ndim, self.shape, sp, v, dt, nt, self.opts,
                                       stream)

    def close(self):
        if getattr(self, "handle", None):
            fwi_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        return fwi_model_info(self.handle)

    def update_velocity(self, v, stream=None):
        fwi_update_velocity(self.handle, v.contiguous() if hasattr(v, "contiguous") else v,
                            stream)

    def forward(self, acq: Acquisition, wavelets, traces=None, final_state=False,
                stream=None):
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        if traces is None:
            traces = torch.empty((acq.nshots, self.nt, acq.nrec), dtype=torch.float32,
                                 device=dev)
        fin = None
        if final_state:
            cs = self.info()["computed"]
            fin = torch.empty((acq.nshots, 2, cs[0], cs[1], cs[2]), dtype=torch.float32,
                              device=dev)
        fwi_forward(self.handle, acq.c, wavelets, traces, fin, stream)
        return (traces, fin) if final_state else traces

    def gradient(self, acq: Acquisition, wavelets, d_obs, want64=False, stream=None):
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        phys = self.shape if self.ndim == 3 else (self.shape[0], self.shape[2])
        misfit = torch.zeros(1, dtype=torch.float64, device=dev)
        grad = torch.empty(phys, dtype=torch.float32, device=dev)
        g64 = torch.empty(phys, dtype=torch.float64, device=dev) if want64 else None
        fwi_adjoint_gradient(self.handle, acq.c, wavelets, d_obs, misfit, grad, g64, stream)
        return (misfit, grad, g64) if want64 else (misfit, grad)

    def source_adjoint(self, acq: Acquisition, y, stream=None):
        import torch
        x = torch.empty((acq.nshots, self.nt), dtype=torch.float32, device=y.device)
        fwi_source_adjoint(self.handle, acq.c, y, x, stream)
        return x


def _autograd_function():
    import torch

    class WaveFwi(torch.autograd.Function):
        """misfit = WaveFwi.apply(v, model, acq, wavelets, d_obs)

        Forward: installs v in the model and runs ``fwi_adjoint_gradient`` once, which
        returns the misfit (Eq. 1) and its exact gradient; the gradient is kept for the
        backward pass, which only scales it by the incoming gradient.  v is the physical
        velocity grid (float32, CUDA)."""

        @staticmethod
        def forward(ctx, v, model, acq, wavelets, d_obs):
            model.update_velocity(v.detach().contiguous())
            phi, grad = model.gradient(acq, wavelets, d_obs)
            ctx.save_for_backward(grad)
            return phi.to(torch.float32).reshape(())

        @staticmethod
        def backward(ctx, gout):
            (grad,) = ctx.saved_tensors
            return gout * grad, None, None, None, None

    return WaveFwi


_wavefwi = None


def __getattr__(name):
    global _wavefwi
    if name == "WaveFwi":
        if _wavefwi is None:
            _wavefwi = _autograd_function()
        return _wavefwi
    raise AttributeError(name)
