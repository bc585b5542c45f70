"""Differentiable time integration: ``torch.autograd`` over K time steps of
the CUDA path, with the discrete adjoint of ``swdg_step_vjp`` and
checkpointing.

    zeta, qx, qy, c = adjoint.solve(ctx, zeta0, qx0, qy0, c0, manning, delta,
                                    nsteps=200, checkpoint_every=20)
    loss(zeta, ...).backward()   # gradients reach manning, delta and the start state

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

import torch

from . import swdg


class _Spec:
    def __init__(self, ctx, nsteps, dt, t0, every):
        self.ctx, self.nsteps, self.dt, self.t0, self.every = ctx, nsteps, dt, t0, every


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
        dts, ckpt = [], {}
        for i in range(spec.nsteps):
            if i % spec.every == 0:
                ckpt[i] = (ctx.get_state(_empty_state(ctx, zeta)), t)
            dt = spec.dt[i] if isinstance(spec.dt, (list, tuple)) else spec.dt
            t = ctx.step(1, dt, t)
            dts.append(ctx.clock()[1])
        out = ctx.get_state(_empty_state(ctx, zeta))
        fctx.spec, fctx.dts, fctx.ckpt = spec, dts, ckpt
        fctx.save_for_backward(manning, delta)
        return tuple(out)

    @staticmethod
    def backward(fctx, gz, gqx, gqy, gc):
        spec, dts, ckpt = fctx.spec, fctx.dts, fctx.ckpt
        manning, delta = fctx.saved_tensors
        ctx = spec.ctx
        dev = manning.device
        ub = [g.contiguous() if g is not None else
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
                r = ctx.step_vjp(ub, slot=i - i0)
                ub = [r["zeta"], r["qx"], r["qy"], r["c"]]
                nb += r["manning"]
                db += r["delta"]
        return nb, db, ub[0], ub[1], ub[2], ub[3], None


def solve(ctx: swdg.Context, zeta, qx, qy, c, manning, delta, nsteps, dt=-1.0, t0=0.0,
          checkpoint_every=20):
    """K = nsteps time steps from (zeta, qx, qy, c) at t0 with Manning
    coefficients ``manning`` and bathymetry offsets ``delta``; ``dt`` < 0: the
    CFL step, a number: a fixed step, a sequence: the step of each step.
    Returns the final (zeta, qx, qy, c), differentiable with respect to every
    tensor argument.  The context is left at a state of the backward pass."""
    if checkpoint_every < 1:
        raise ValueError("checkpoint_every must be >= 1")
    return _Solve.apply(manning, delta, zeta, qx, qy, c,
                        _Spec(ctx, int(nsteps), dt, float(t0), int(checkpoint_every)))
