"""Discrete adjoint of the time step on the GPU (swdg_step_record +
swdg_step_vjp) against the step adjoint oracle (autograd of the pinned
PyTorch step along the forward's path): the cotangents of the start state,
the Manning coefficients and the bathymetry offsets after one and two fixed
steps, within 1e-9 of their scale; modes S and P, r = 2, 3, a wet-dry r_K = 0
cell, a 2:1 forest."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from oracle.torch_step import TorchStep, step_vjp
from paper_2505_18743_gb300 import swdg

import test_oracle_step_adjoint as SA

pytestmark = pytest.mark.gpu

TOL = 1e-9
KEYS = ("zeta", "qx", "qy", "c", "manning", "delta")


@pytest.fixture(scope="module", autouse=True)
def _build():
    import torch
    assert torch.cuda.is_available()
    from paper_2505_18743_gb300 import build as B
    from oracle import oracle
    B.build()
    oracle.build()


def gpu_vjp(wl, cot, dt, nsteps):
    """reverse over nsteps fixed steps, re-running each step from its stored start"""
    ctx = swdg.Context.from_workload(wl)
    starts, t = [], 0.0
    for _ in range(nsteps):
        starts.append((ctx.get_state(), t))
        t = ctx.step(1, dt, t)
    nb = np.zeros(wl.mesh.n)
    db = np.zeros(wl.mesh.n)
    ub = cot
    for state, t0 in reversed(starts):
        ctx.set_state(*state)
        ctx.step_record(dt, t0)
        r = ctx.step_vjp(ub)
        ub = [r["zeta"], r["qx"], r["qy"], r["c"]]
        nb += r["manning"]
        db += r["delta"]
    ctx.close()
    return ub + [nb, db]


@pytest.mark.parametrize("nsteps", [1, 2])
@pytest.mark.parametrize("case", sorted(SA.CASES))
def test_step_vjp_matches_the_step_adjoint_oracle(case, nsteps):
    wl = SA.CASES[case]()
    dt = SA.fixed_dt(wl)
    n, nd = wl.mesh.n, (wl.degree + 1) ** 2
    rng = np.random.default_rng(21)
    cot = [rng.standard_normal((n, nd)) for _ in range(4)]
    ref = step_vjp(TorchStep(wl), wl.state(), wl.manning, np.zeros(n), cot, 0.0, dt, nsteps)
    got = gpu_vjp(wl, cot, dt, nsteps)
    errs = {}
    for key, a, b in zip(KEYS, got, ref):
        errs[key] = float(np.abs(a - b).max()) / max(float(np.abs(b).max()), 1e-300)
    assert max(errs.values()) <= TOL, errs


def test_step_record_rejects_what_it_cannot_differentiate():
    wl = SA.CASES["beach_r2"]()
    ctx = swdg.Context.from_workload(wl)
    with pytest.raises(swdg.SwdgError) as e:
        ctx.step_vjp([np.zeros((wl.mesh.n, 9))] * 4)
    assert e.value.code == swdg.SWDG_ESTATE
    with pytest.raises(swdg.SwdgError):
        ctx.step_record(-1.0, 0.0)
    c32 = swdg.Context.from_workload(wl, precision=1)
    with pytest.raises(swdg.SwdgError):
        c32.step_record(1.0, 0.0)
