"""FWI outer iteration (Sec. 1: predict data, measure the misfit, update the model,
repeat until the misfit is small) on top of the library's misfit and gradient.

The paper names the loop but no optimiser; this is projected steepest descent with a
backtracking (Armijo) line search and a box constraint on velocity.  The step is taken
along the gradient scaled to a fixed largest velocity change, so the first trial step
has a physical size (`max_dv` m/s) whatever the misfit's units.
"""
from __future__ import annotations

from typing import Callable, List, Tuple


def descend(v0, misfit_and_grad: Callable, iters: int = 5, max_dv: float = 50.0,
            vmin: float = 1500.0, vmax: float = 4500.0, shrink: float = 0.5,
            max_tries: int = 6, c1: float = 1e-4, mask=None) -> Tuple[object, List[float]]:
    """Minimises phi(v) from v0.  `misfit_and_grad(v)` returns (phi, grad) for a torch
    tensor or numpy array v; `v` keeps its type.  Returns (v, misfit history).  A trial
    step alpha * d with d = -grad * (max_dv / max|grad|) (cells held at a bound by the
    descent left out: projected gradient) is accepted when
    phi(clip(v + alpha d)) <= phi(v) + c1 * alpha * <grad, d>; otherwise alpha halves (at
    most max_tries times, then the loop stops).  Each line search starts from twice the
    previously accepted alpha (at most 1).  `mask` (same shape as v, values in [0, 1])
    mutes the update where it is 0: the usual mute of the cells next to the sources and
    receivers, where the gradient's near-field peaks would otherwise set the step size
    and leave the rest of the model almost unchanged."""
    v = v0.clone() if hasattr(v0, "clone") else v0.copy()
    phi, g = misfit_and_grad(v)
    hist = [float(phi)]
    alpha0 = 1.0
    for _ in range(iters):
        # projected direction: cells at a bound that the descent would push outward stay
        blocked = ((v <= vmin) & (g > 0)) | ((v >= vmax) & (g < 0))
        gp = g * (~blocked)
        if mask is not None:
            gp = gp * mask
        gmax = float(abs(gp).max())
        if gmax == 0.0:
            break
        d = -gp * (max_dv / gmax)
        slope = float((g * d).sum())          # directional derivative, negative
        alpha, accepted = alpha0, False
        for _ in range(max_tries):
            trial = v + alpha * d
            trial = trial.clamp(vmin, vmax) if hasattr(trial, "clamp") else trial.clip(vmin, vmax)
            phi_t, g_t = misfit_and_grad(trial)
            if float(phi_t) <= float(phi) + c1 * alpha * slope:
                v, phi, g, accepted = trial, phi_t, g_t, True
                break
            alpha *= shrink
        if not accepted:
            break
        alpha0 = min(1.0, 2.0 * alpha)
        hist.append(float(phi))
    return v, hist


def gpu_evaluator(model, acq, wavelets, d_obs):
    """misfit_and_grad for `descend` through the library's autograd Function: the
    forward installs v and evaluates the misfit and its gradient in one call."""
    from . import fwi

    def f(v):
        vv = v.detach().clone().requires_grad_(True)
        phi = fwi.WaveFwi.apply(vv, model, acq, wavelets, d_obs)
        phi.backward()
        return phi.item(), vv.grad.detach()

    return f


def _smooth(v, cells: float):
    """Gaussian-smoothed copy of a velocity grid (standard deviation `cells`): the usual
    starting model of an FWI run, which keeps the kinematics and loses the interfaces."""
    from scipy.ndimage import gaussian_filter
    return gaussian_filter(v.astype("float64"), sigma=cells, mode="nearest").astype("float32")


def faulted_2d_start(w, smooth_cells: float, mute_rows: int):
    """Starting model and update mask for an FWI run on a faulted 2-D workload: the true
    model smoothed by a Gaussian of `smooth_cells` cells, and a mask that is 0 on the
    first `mute_rows` rows (sources and receivers lie there) and ramps to 1 over the next
    10 rows.  Both numpy float32."""
    import numpy as np
    nz, nx = w.shape
    v0 = _smooth(w.v, smooth_cells)
    mask = np.ones((nz, nx), dtype=np.float32)
    mask[:mute_rows] = 0.0
    mask[mute_rows:mute_rows + 10] = np.linspace(0.0, 1.0, 10, dtype=np.float32)[:, None]
    return v0, mask


def model_error(v, v_true) -> float:
    """||v - v_true|| / ||v_true - mean(v_true)||"""
    import numpy as np
    vt = np.asarray(v_true, dtype=np.float64)
    return float(np.linalg.norm(np.asarray(v, dtype=np.float64) - vt) / np.linalg.norm(vt - vt.mean()))


def run_faulted_2d(iters: int = 8, nz: int = 400, nx: int = 1024, nt: int = 3000,
                   nshots: int = 64, smooth_cells: float = 12.0, max_dv: float = 40.0,
                   mute_rows: int = 20, device: str = "cuda:0", return_model: bool = False) -> dict:
    """FWI of the faulted 2-D model with a salt ellipse (all shots in one batched gradient
    call per evaluation, through the autograd Function): observed data from the true
    model, a smoothed starting model, rows next to the sources and receivers muted.
    Returns the misfit history, the relative model error before and after, the
    correlation of the update with the true model's departure from the start, and the
    seconds spent per misfit-and-gradient evaluation (plus the final model as a numpy
    array under "v" when `return_model`)."""
    import time

    import numpy as np
    import torch

    from . import fwi, synth

    w = synth.faulted_2d(nz=nz, nx=nx, nt=nt, nshots=nshots)
    dev = torch.device(device)
    acq = fwi.Acquisition(w.src, w.rec)
    wav = torch.from_numpy(w.wavelets()).to(dev)
    obs = fwi.FwiModel(torch.from_numpy(w.v).to(dev), w.h, w.dt, w.nt, order=w.order,
                       sponge_vref=4500.0)
    d_obs = obs.forward(acq, wav)
    obs.close()
    v0, mask = faulted_2d_start(w, smooth_cells, mute_rows)
    m = fwi.FwiModel(torch.from_numpy(v0).to(dev), w.h, w.dt, w.nt, order=w.order,
                     snap_dtype=w.snap_dtype, sponge_vref=4500.0)
    evals = [0]
    f0 = gpu_evaluator(m, acq, wav, d_obs)

    def f(v):
        evals[0] += 1
        return f0(v)

    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    v, hist = descend(torch.from_numpy(v0).to(dev), f, iters=iters, max_dv=max_dv,
                      mask=torch.from_numpy(mask).to(dev))
    torch.cuda.synchronize(dev)
    secs = time.perf_counter() - t0
    m.close()
    v = v.cpu().numpy()
    dv, dt_ = (v - v0).astype(np.float64), (w.v - v0).astype(np.float64)
    corr = float((dv * dt_).sum() / max(np.linalg.norm(dv) * np.linalg.norm(dt_), 1e-300))
    out = {"workload": w.name, "nt": nt, "iterations": len(hist) - 1, "evaluations": evals[0],
           "misfit": hist, "model_error_start": model_error(v0, w.v),
           "model_error_end": model_error(v, w.v), "update_correlation": corr,
           "seconds": secs, "seconds_per_evaluation": secs / max(evals[0], 1),
           "shots_per_second": nshots * evals[0] / secs}
    if return_model:
        out["v"] = v
    return out


if __name__ == "__main__":
    import argparse
    import json

    ap = argparse.ArgumentParser(description="FWI of the 400 x 1024 faulted 2-D model, 64 shots")
    ap.add_argument("--iters", type=int, default=8)
    ap.add_argument("--nt", type=int, default=3000)
    a = ap.parse_args()
    print(json.dumps(run_faulted_2d(iters=a.iters, nt=a.nt)))
