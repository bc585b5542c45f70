"""Differentiable time integration: ``torch.autograd`` over K time steps of
the CUDA path, with the discrete adjoint of ``swdg_step_vjp`` and
checkpointing.

    zeta, qx, qy, c = adjoint.solve(ctx, zeta0, qx0, qy0, c0, manning, delta,
                                    nsteps=200, checkpoint_every=20)
    loss(zeta, ...).backward()   # gradients reach manning, delta and the start state

    # or a loss over time: G [nsteps, n_gauges] = zeta at the gauges after each step
    *state, G = adjoint.solve(..., gauges=xy)
    ((G - G_truth) ** 2).sum().backward()

``manning`` (Manning coefficient per cell) and ``delta`` (bathymetry offset
per cell: every depth of cell K deepened by delta_K) and the start state are
CUDA float64 tensors.  The forward run keeps the state every
``checkpoint_every`` steps and the time step of every step (the CFL step,
``dt < 0``, or a fixed one); the backward pass re-runs each block of steps
from its checkpoint once, keeping a record of every step of the block, then
pulls the steps back in reverse order from their records.
The time steps and every discrete decision of the forward run are held fixed
in the adjoint (the derivative along the forward's path).  All arithmetic
runs in the library's kernels; this module only orders the calls.
"""
from __future__ import annotations

import numpy as np
import torch

from . import swdg


class _Spec:
    def __init__(self, ctx, nsteps, dt, t0, every, gauges):
        self.ctx, self.nsteps, self.dt, self.t0, self.every = ctx, nsteps, dt, t0, every
        self.gauges = gauges  # [ng, 2] host array or None


def _clone(state):
    return [s.clone() for s in state]


def _empty_state(ctx, like):
    return [torch.empty((ctx.n, ctx.nd), dtype=torch.float64, device=like.device) for _ in range(4)]


class _Solve(torch.autograd.Function):
    @staticmethod
    def forward(fctx, manning, delta, zeta, qx, qy, c, spec):
        ctx = spec.ctx
        ctx.set_manning(manning.contiguous())
        ctx.set_bathymetry_offset(delta.contiguous())
        ctx.set_state(zeta.contiguous(), qx.contiguous(), qy.contiguous(), c.contiguous())
        t = spec.t0
        dts, ckpt, obs = [], {}, []
        for i in range(spec.nsteps):
            if i % spec.every == 0:
                ckpt[i] = (ctx.get_state(_empty_state(ctx, zeta)), t)
            dt = spec.dt[i] if isinstance(spec.dt, (list, tuple)) else spec.dt
            t = ctx.step(1, dt, t)
            dts.append(ctx.clock()[1])
            if spec.gauges is not None:
                obs.append(ctx.gather_gauges(spec.gauges))
        out = ctx.get_state(_empty_state(ctx, zeta))
        ng = 0 if spec.gauges is None else len(spec.gauges)
        G = torch.from_numpy(np.stack(obs) if obs else np.zeros((spec.nsteps, 0)))
        G = G.to(zeta.device, torch.float64).reshape(spec.nsteps, ng)
        fctx.spec, fctx.dts, fctx.ckpt = spec, dts, ckpt
        fctx.save_for_backward(manning, delta)
        return tuple(out) + (G,)

    @staticmethod
    def backward(fctx, gz, gqx, gqy, gc, gG):
        spec, dts, ckpt = fctx.spec, fctx.dts, fctx.ckpt
        gGh = None
        if spec.gauges is not None and gG is not None:
            gGh = gG.detach().to("cpu", torch.float64).numpy()
        manning, delta = fctx.saved_tensors
        ctx = spec.ctx
        dev = manning.device
        ub = [g.clone(memory_format=torch.contiguous_format) if g is not None else
              torch.zeros((ctx.n, ctx.nd), dtype=torch.float64, device=dev)
              for g in (gz, gqx, gqy, gc)]
        nb = torch.zeros(ctx.n, dtype=torch.float64, device=dev)
        db = torch.zeros(ctx.n, dtype=torch.float64, device=dev)
        ctx.set_manning(manning.contiguous())
        ctx.set_bathymetry_offset(delta.contiguous())
        ctx.adjoint_slots(min(spec.every, spec.nsteps))
        for i0 in sorted(ckpt, reverse=True):
            i1 = min(i0 + spec.every, spec.nsteps)
            state, t = ckpt[i0]
            ctx.set_state(*state)
            for i in range(i0, i1):  # re-run the block, recording every step
                t = ctx.step_record(dts[i], t, slot=i - i0)
            for i in reversed(range(i0, i1)):
                if gGh is not None and gGh[i].any():
                    # the gauge observations taken after step i
                    ctx.gauges_vjp(spec.gauges, gGh[i], ub[0])
                r = ctx.step_vjp(ub, slot=i - i0)
                ub = [r["zeta"], r["qx"], r["qy"], r["c"]]
                nb += r["manning"]
                db += r["delta"]
        return nb, db, ub[0], ub[1], ub[2], ub[3], None


def solve(ctx: swdg.Context, zeta, qx, qy, c, manning, delta, nsteps, dt=-1.0, t0=0.0,
          checkpoint_every=20, gauges=None):
    """K = nsteps time steps from (zeta, qx, qy, c) at t0 with Manning
    coefficients ``manning`` and bathymetry offsets ``delta``; ``dt`` < 0: the
    CFL step, a number: a fixed step, a sequence: the step of each step.
    Returns the final (zeta, qx, qy, c), and with ``gauges`` (xy [ng, 2]) also
    G [nsteps, ng], zeta at the gauges after each step (swdg_gather_gauges);
    all differentiable with respect to every tensor argument.  The context is
    left at a state of the backward pass."""
    if checkpoint_every < 1:
        raise ValueError("checkpoint_every must be >= 1")
    xy = None if gauges is None else np.ascontiguousarray(gauges, dtype=np.float64)
    if xy is not None and (xy.ndim != 2 or xy.shape[1] != 2):
        raise ValueError("gauges must be an [ng, 2] array of points")
    out = _Solve.apply(manning, delta, zeta, qx, qy, c,
                       _Spec(ctx, int(nsteps), dt, float(t0), int(checkpoint_every), xy))
    return out if xy is not None else out[:4]
