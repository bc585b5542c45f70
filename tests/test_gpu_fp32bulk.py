"""FP32-bulk precision (swdg_config.precision = 1) against the FP64 oracle.

The momentum, friction and flux arithmetic of the residual runs in FP32
(with the elevation's gradient, which only the FP32 pressure product
uses), so those results carry FP32 error (bounded here, and stated per
result); the elevation's values, the sub-grid integrals, the hydrostatic
reconstruction (including the depth jump h*- - h*+), the continuity and
tracer test integrals and every stage solve stay FP64, so the lake at rest,
water mass and tracer mass hold to FP64 round-off as in the plain path.  A
constant tracer (c = 1) is kept to FP32 level only: once c is not bitwise
constant its FP32 interpolation departs from 1 by ~1e-7.
"""
import numpy as np
import pytest

from helpers import rel_inf, residual_errors
from oracle.oracle import Oracle
from paper_2505_18743_gb300 import swdg
from paper_2505_18743_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# FP32 result error bounds (relative to the field's max magnitude)
RES_TOL_FP32 = 1e-5
STATE_TOL_FP32 = 1e-5
CWC_TOL_FP32 = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _build():
    import torch
    assert torch.cuda.is_available()
    from paper_2505_18743_gb300 import build as B
    from oracle import oracle
    B.build()
    oracle.build()


def island(degree=2, amp=0.5):
    wl = W.closed_basin(degree=degree)
    npx = wl.raster.z.shape[0]
    xc = (np.arange(npx) + 0.5) * wl.raster.dx
    X, Y = np.meshgrid(xc, xc)
    wl.raster.z = wl.raster.z - 8.0 * np.exp(-((X - 500) ** 2 + (Y - 500) ** 2) / 150.0 ** 2)
    Xn, Yn = W.nodal_coordinates(wl.mesh, degree)
    wl.zeta = amp * np.exp(-((Xn - 300) ** 2 + (Yn - 500) ** 2) / 100.0 ** 2)
    wl.c = np.ones_like(wl.zeta)
    wl.tableau = 0
    wl.cfl = 0.9 * {1: 1 / 6, 2: 1 / 12, 3: 1 / 20}[degree] / (2 - np.sqrt(2))
    return wl


@pytest.mark.parametrize("degree", [1, 2, 3])
def test_fp32bulk_residual_within_fp32_error(degree):
    wl = W.tidal_beach(window=(236, 120, 12, 8), degree=degree, pix=16)
    Xn, Yn = W.nodal_coordinates(wl.mesh, degree)
    wl.zeta = 0.3 * np.sin(Xn / 400.0) * np.cos(Yn / 300.0)
    wl.qx = 0.2 * np.cos(Yn / 200.0) * np.ones_like(Xn)
    ctx = swdg.Context.from_workload(wl, precision=1)
    ora = Oracle.from_workload(wl)
    rg, ro = ctx.residual(1000.0), ora.residual(1000.0)
    errs = residual_errors(rg, ro)  # each field against its own scale
    assert max(errs.values()) <= RES_TOL_FP32, errs


def test_fp32bulk_lake_at_rest_is_exact():
    wl = W.lake_at_rest_bump(n=8, pix=4, degree=2, submerged=False)
    ora = Oracle.from_workload(wl)
    z = ora.lake_at_rest(0.0)
    zero = np.zeros_like(z)
    wl.zeta, wl.qx, wl.qy, wl.c = z, zero, zero.copy(), np.ones_like(z)
    ctx = swdg.Context.from_workload(wl, precision=1)
    for k, v in ctx.residual(0.0).items():
        assert np.abs(v).max() < 1e-13 * 9.81, k
    ctx.step(25, -1.0, 0.0)
    zg, qxg, qyg, cg = ctx.get_state()
    assert np.abs(zg - z).max() < 1e-13 and np.abs(qxg).max() < 1e-13 and np.abs(qyg).max() < 1e-13


def test_fp32bulk_mass_tracer_and_cwc_at_fp64_roundoff():
    wl = island(2)
    ctx = swdg.Context.from_workload(wl, precision=1)
    d0 = ctx.diagnostics()
    ctx.step(40, -1.0, 0.0)
    d1 = ctx.diagnostics()
    assert abs(d1["mass"] - d0["mass"]) <= 1e-13 * d0["mass"]
    assert abs(d1["tracer_mass"] - d0["tracer_mass"]) <= 1e-13 * d0["tracer_mass"]
    assert np.abs(ctx.get_state()[3] - 1.0).max() < CWC_TOL_FP32
    assert d1["positivity_violations"] == 0


def test_fp32bulk_steps_within_fp32_error_of_oracle():
    wl = W.tidal_beach(window=(0, 120, 12, 8))
    wl.zeta = 0.2 * np.ones_like(wl.zeta)
    ctx = swdg.Context.from_workload(wl, precision=1)
    ora = Oracle.from_workload(wl)
    ctx.step(20, -1.0, 1000.0)
    ora.step(20, -1.0, 1000.0)
    sg, so = ctx.get_state(), ora.get_state()
    qscale = max(float(np.abs(so[1]).max()), float(np.abs(so[2]).max()))  # discharge magnitude
    for name, a, b in zip(("zeta", "qx", "qy", "c"), sg, so):
        floor = 1.0 if name in ("zeta", "c") else qscale
        assert rel_inf(a, b, floor=floor) <= STATE_TOL_FP32, name


def test_fp32bulk_state_copy_follows_every_state_write():
    """FP32-bulk contexts keep an FP32 copy of the state for the FP32 face and
    residual arithmetic; it must follow every write of the state.  The
    autotuner steps on the context's own state and restores it: the residual
    after it equals the one before bit for bit.  A stepped context and a
    fresh one given the stepped state agree bit for bit, and so does the
    first context after a new state upload."""
    wl = island(3)
    ctx = swdg.Context.from_workload(wl, precision=1)
    r0 = ctx.residual(0.0)
    ctx.autotune(repeats=1)
    r1 = ctx.residual(0.0)
    for k in r0:
        assert np.array_equal(r0[k], r1[k]), k
    ctx.step(3, -1.0, 0.0)
    fresh = swdg.Context.from_workload(wl, precision=1)
    fresh.set_state(*ctx.get_state())
    rg, rf = ctx.residual(5.0), fresh.residual(5.0)
    for k in rg:
        assert np.array_equal(rg[k], rf[k]), k
    ctx.set_state(*wl.state())
    r2 = ctx.residual(0.0)
    for k in r0:
        assert np.array_equal(r0[k], r2[k]), k
