"""Leapfrog dynamics on the kd-tree FMM force, and its derivative.

* `integrate` -- kick-drift-kick leapfrog with the tree rebuilt every step,
  recording the centre of mass and the total force sum m a after each step
  (the drift the paper analyses in Sec. 4).  Kick, drift and both reductions
  run in the library's kernels; nothing is differentiated.
* `FmmAccel` -- one force evaluation as a torch.autograd.Function: forward is
  tree build + evaluation, backward the library's adjoint through the same
  tree and interaction lists (kdfmm_fmm_accel_vjp).
* `leapfrog` -- the same integrator in differentiable form, with reentrant
  checkpointing: only every k-th state is kept; a segment's trees are rebuilt
  when its backward pass runs, so at most one segment of trees is alive.
"""
from __future__ import annotations

import torch
import torch.utils.checkpoint as ckpt

from . import native


# Handles not in use, per (device, parameters).  A handle keeps its buffers
# and list capacities between builds, so taking one from here spares an
# evaluation the allocations and the first-call sizing of a new handle; an
# evaluation whose backward may still run keeps its handle (the adjoint needs
# its tree and lists) until then.
_FREE: dict = {}
_FREE_MAX = 16


def _key(params: dict):
    return (torch.cuda.current_device(), tuple(sorted(params.items())))


def _take(params: dict):
    free = _FREE.get(_key(params))
    return free.pop() if free else native.KdFmm(**params)


def _give(params: dict, f) -> None:
    free = _FREE.setdefault(_key(params), [])
    if len(free) < _FREE_MAX:
        free.append(f)


class FmmAccel(torch.autograd.Function):
    """a = FMM acceleration of particles x (n, 3) with masses m (n,) and
    smoothing lengths h (n,) or None; `params` the kdfmm parameters."""

    @staticmethod
    def forward(ctx, x, m, h, params: dict):
        f = _take(params)
        f.build(x.detach().contiguous(), m.detach().contiguous(),
                None if h is None else h.detach().contiguous())
        a, _ = f.accel(want_phi=False)
        if ctx.needs_input_grad[0] or ctx.needs_input_grad[1]:
            ctx.f, ctx.params = f, params
        else:                                   # no backward will come
            ctx.f = None
            _give(params, f)
        return a

    @staticmethod
    def backward(ctx, a_bar):
        f, ctx.f = ctx.f, None
        x_bar, m_bar = f.vjp(a_bar.contiguous())
        _give(ctx.params, f)
        return x_bar, (m_bar if ctx.needs_input_grad[1] else None), None, None


def fmm_accel(x, m, h=None, **params):
    return FmmAccel.apply(x, m, h, params)


def _kdk(x, v, a, m, h, dt, params):
    v_half = v + (0.5 * dt) * a
    x1 = x + dt * v_half
    a1 = FmmAccel.apply(x1, m, h, params)
    return x1, v_half + (0.5 * dt) * a1, a1


def leapfrog(x0, v0, m, h=None, *, steps: int, dt: float, checkpoint_every: int = 10, **params):
    """Differentiable KDK leapfrog; returns the final (x, v, a).  Gradients
    flow to x0 and v0 (m and h are held fixed).  With checkpoint_every > 0
    only segment boundaries are stored during the forward pass."""
    a = FmmAccel.apply(x0, m, h, params)
    x, v = x0, v0
    s = 0
    while s < steps:
        nseg = min(checkpoint_every if checkpoint_every > 0 else steps, steps - s)

        def segment(x, v, a, nseg=nseg):
            for _ in range(nseg):
                x, v, a = _kdk(x, v, a, m, h, dt, params)
            return x, v, a

        if checkpoint_every > 0 and torch.is_grad_enabled():
            x, v, a = ckpt.checkpoint(segment, x, v, a, use_reentrant=True)
        else:
            x, v, a = segment(x, v, a)
        s += nseg
    return x, v, a


def centre_of_mass(x, m):
    return (m[:, None] * x).sum(0) / m.sum()


def integrate(x, v, m, h=None, *, steps: int, dt: float, record_every: int = 1, **params):
    """KDK leapfrog in place on device tensors x, v (n, 3); returns a dict of
    host arrays: step, com (centre of mass), F (sum m a) per recorded step."""
    import numpy as np
    f = native.KdFmm(**params)
    n = x.shape[0]
    a = torch.empty((n, 3), dtype=torch.float64, device=x.device)
    out = torch.empty(3, dtype=torch.float64, device=x.device)
    mom = torch.empty(3, dtype=torch.float64, device=x.device)
    M = float(m.sum())
    steps_rec, com, F = [], [], []

    def record(k):
        native.total_momentum(m, x, mom)      # sum m x
        native.total_momentum(m, a, out)      # sum m a
        c, g = mom.cpu().numpy() / M, out.cpu().numpy()
        steps_rec.append(k)
        com.append(c)
        F.append(g)

    f.build(x, m, h)
    f.accel(a, None, want_phi=False)
    record(0)
    for k in range(1, steps + 1):
        native.kick_drift(x, v, a, 0.5 * dt, dt)
        f.build(x, m, h)
        f.accel(a, None, want_phi=False)
        native.kick_drift(x, v, a, 0.5 * dt, 0.0)
        if k % record_every == 0 or k == steps:
            record(k)
    return {"step": np.array(steps_rec), "com": np.array(com), "F": np.array(F)}
