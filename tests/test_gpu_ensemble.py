"""Batched ensembles and launch shapes on the GPU (through the C-ABI).

An ensemble is one context whose mesh is the disjoint union of independent
members; each member keeps its own CFL step, clock, tide and raster while
every kernel of a step is one launch over all members.  Because each cell's
arithmetic is the same as in a stand-alone context (the CFL maximum is an
order-independent max), a member of an ensemble must reproduce its
stand-alone context bit for bit, and the stand-alone context is in turn held
to the oracle.  Launch shapes (block size, persistent or full grid) must not
change a single bit either.
"""
import ctypes

import numpy as np
import pytest

from helpers import rel_inf
from oracle.oracle import Oracle
from paper_2505_18743_gb300 import swdg
from paper_2505_18743_gb300 import workloads as W

pytestmark = pytest.mark.gpu

STATE_TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _build():
    import torch
    assert torch.cuda.is_available()
    from paper_2505_18743_gb300 import build as B
    from oracle import oracle
    B.build()
    oracle.build()


def small_members(m=4, degree=2, sizes=(6, 8, 10), pix=8):
    # full 20 km beaches on coarse meshes: shoreline, channels and tide in each
    return W.beach_ensemble(members=m, sizes=sizes, pix=pix, degree=degree)


def same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


@pytest.mark.parametrize("precision", [0, 1])
def test_members_reproduce_standalone_contexts_bitwise(precision):
    wls = small_members(4)
    assert len({w.mesh.n for w in wls}) > 1 and len({w.boundaries[0][2] for w in wls}) == 4
    ens = swdg.Ensemble.from_workloads(wls, precision=precision)
    ens.step(12)
    t_ens, dt_ens = ens.times()
    for m, wl in enumerate(wls):
        ctx = swdg.Context.from_workload(wl, precision=precision)
        t = ctx.step(12, -1.0, 0.0)
        assert same(ens.member_state(m), ctx.get_state()), m
        assert t_ens[m] == t
        assert dt_ens[m] == ctx.diagnostics()["dt"]
        ctx.close()
    # members took different steps
    assert len(set(dt_ens.tolist())) == len(wls)


def test_members_match_the_oracle():
    wls = small_members(3, sizes=(6, 8))
    ens = swdg.Ensemble.from_workloads(wls)
    ens.step(8)
    t_ens, _ = ens.times()
    for m, wl in enumerate(wls):
        ora = Oracle.from_workload(wl)
        t = ora.step(8, -1.0, 0.0)
        assert abs(t - t_ens[m]) <= 1e-12 * t
        for name, a, b in zip(("zeta", "qx", "qy", "c"), ens.member_state(m), ora.get_state()):
            floor = 1.0 if name in ("zeta", "c") else 1e-3
            assert rel_inf(a, b, floor=floor) <= STATE_TOL, (m, name)


def test_member_diagnostics_and_clocks():
    wls = small_members(3)
    ens = swdg.Ensemble.from_workloads(wls)
    d0 = ens.member_diagnostics()
    ens.set_times([0.0, 100.0, 200.0])
    ens.step(5)
    t, dt = ens.times()
    assert np.all(t > np.array([0.0, 100.0, 200.0])) and np.all(dt > 0)
    d1 = ens.member_diagnostics()
    tot = ens.diagnostics()
    assert abs(sum(d["mass"] for d in d1) - tot["mass"]) <= 1e-13 * tot["mass"]
    for m, wl in enumerate(wls):
        ctx = swdg.Context.from_workload(wl)
        dm = ctx.diagnostics()
        assert dm["mass"] == d0[m]["mass"] and dm["tracer_mass"] == d0[m]["tracer_mass"]
        assert d1[m]["t"] == t[m] and d1[m]["dt"] == dt[m]
        ctx.close()


def test_member_gauges():
    wls = small_members(2, sizes=(8,))
    ens = swdg.Ensemble.from_workloads(wls)
    ens.step(3)
    xy = np.array([[1000.0, 5000.0], [17000.0, 12000.0], [-5.0, 0.0]])
    for m, wl in enumerate(wls):
        ctx = swdg.Context.from_workload(wl)
        ctx.step(3, -1.0, 0.0)
        a, b = ens.gather_gauges_member(m, xy), ctx.gather_gauges(xy)
        assert np.array_equal(a[:2], b[:2]) and np.isnan(a[2]) and np.isnan(b[2])
        ctx.close()


def test_ensemble_argument_checks():
    wls = small_members(2, sizes=(6,))
    ens = swdg.Ensemble.from_workloads(wls)
    n = ens.n
    L = swdg.load()
    # a member boundary that cuts a face, a member without cells, bad ends
    for first in ([0, 10, n], [0, 36, 36, n], [0, 36, n - 1], [1, 36, n]):
        f = np.asarray(first, dtype=np.int64)
        assert L.swdg_set_members(ens.h, len(f) - 1, f.ctypes.data_as(ctypes.c_void_p)) \
            == swdg.SWDG_EINVAL, first
    # the ensemble is unchanged by the rejected calls; t_inout is refused
    t = ctypes.c_double(0.0)
    assert L.swdg_step(ens.h, 1, -1.0, ctypes.byref(t)) == swdg.SWDG_EINVAL
    assert L.swdg_set_boundary_member(ens.h, 2, 1, swdg.SWDG_BC_TIDE, 1.0, 100.0, 0.0) \
        == swdg.SWDG_EINVAL
    ens.step(1)
    assert ens.times()[0][0] > 0


def test_launch_shapes_do_not_change_results():
    wl = W.tidal_beach(window=(230, 100, 16, 12), degree=3)
    ref = swdg.Context.from_workload(wl)
    t_ref = ref.step(4, -1.0, 0.0)
    s_ref = ref.get_state()
    for wpb in (1, 2, 8):
        for grid in (152, 7, 48):
            ctx = swdg.Context.from_workload(wl)
            for kind in range(4):
                ctx.set_shape(kind, grid, wpb)
            assert ctx.shapes()["stage"] == (grid, wpb)
            t = ctx.step(4, -1.0, 0.0)
            assert t == t_ref and same(ctx.get_state(), s_ref), (wpb, grid)
            ctx.close()
    with pytest.raises(swdg.SwdgError):
        ref.set_shape(1, 10, 16)


def test_autotune_leaves_no_trace_and_keeps_results():
    wls = small_members(4, sizes=(8, 10))
    ens = swdg.Ensemble.from_workloads(wls)
    s0 = ens.get_state()
    t0 = ens.times()[0]
    rep = ens.autotune(repeats=1)
    assert set(rep) == {"begin", "residual", "stage"}
    for grid, wpb, ms in rep.values():
        assert grid >= 1 and wpb in (1, 2, 4, 8) and ms > 0
    assert same(ens.get_state(), s0) and np.array_equal(ens.times()[0], t0)
    ens.step(3)
    plain = swdg.Ensemble.from_workloads(wls)
    plain.step(3)
    assert same(ens.get_state(), plain.get_state())
