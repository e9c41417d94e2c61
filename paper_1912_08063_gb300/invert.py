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
