"""Dynamic h-adaptation on the GPU (swdg_amr_*) against the adaptation
reference (oracle/amr.py) and the C oracle: the refinement indicators of
Sec. 4.4 and Sec. 5, one adaptation (the new mesh, the remapped state to
round-off, the reported Q^n = the change of the total wet mass), and an
adaptive run of the travelling vortex (Sec. 4.4) and of the shoreline
(wet-dry cells, |grad c| indicator) that follows the same chain of steps and
adaptations as the oracle."""
import numpy as np
import pytest

from helpers import Vortex, rel_inf
from oracle.amr import Forest, indicator, remap
from oracle.oracle import Oracle
from paper_2505_18743_gb300 import swdg
from paper_2505_18743_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    import torch
    assert torch.cuda.is_available()
    from paper_2505_18743_gb300 import build as B
    from oracle import oracle
    B.build()
    oracle.build()


def vortex_case(degree=2, N=6):
    v = Vortex()
    F = Forest(2 * N, N, 0.0, 0.0, v.Lx / (2 * N), v.Ly / N, 2, 0.0, (0, 0, 0, 0), (True, True))
    leaves = F.order({(0, i, j) for i in range(2 * N) for j in range(N)})
    mesh = W.Mesh(*F.mesh(leaves))
    ras = W.Raster(np.full((N * 8, 2 * N * 8), v.h0), 0.0, 0.0, v.Lx / (2 * N * 8), v.Ly / (N * 8))
    X, Y = W.nodal_coordinates(mesh, degree)
    h, u, w = v(X, Y, 0.0)
    wl = W.Workload("vortex-amr", degree, mesh, ras, h - v.h0, h * u, h * w, np.ones_like(h),
                    tableau=1, cfl=0.2, eps_vel=1e-3, h_lim=1e-3)
    return wl, F, leaves


def shore_case(degree=1):
    # 20 km beach on 10 x 6 coarse cells of 2 km, 32 px each (62.5 m px), two levels
    rng = np.random.default_rng(20250524)
    z, dx = W.beach_raster(rng, 320, 20000.0)
    z = z[:192]
    F = Forest(10, 6, 0.0, 0.0, 2000.0, 2000.0, 2, 0.0, (1, 0, 0, 0), (False, False))
    leaves = F.order({(0, i, j) for i in range(10) for j in range(6)})
    mesh = W.Mesh(*F.mesh(leaves))
    X, Y = W.nodal_coordinates(mesh, degree)
    zeta = 0.3 * np.ones_like(X)
    c = 0.5 + 0.5 * np.tanh((X - 17000.0) / 400.0)
    zero = np.zeros_like(X)
    wl = W.Workload("shore-amr", degree, mesh, W.Raster(z, 0.0, 0.0, dx, dx), zeta, zero.copy(),
                    zero.copy(), c, tableau=0, cfl=0.1, eps_vel=0.1, h_lim=0.1,
                    boundaries=[(1, W.BC_TIDE, 0.5, 44712.0, 0.0)],
                    manning=np.full(mesh.n, 0.02))
    return wl, F, leaves


def oracle_of(wl, mesh, state, manning):
    o = Oracle(mesh, wl.raster, **wl.config())
    for (tag, kind, amp, per, ph) in wl.boundaries:
        o.set_boundary(tag, kind, amp, per, ph)
    o.set_manning(manning)
    o.set_state(*state)
    return o


def carry(F, old, new, vals):
    idx = {c: k for k, c in enumerate(old)}
    out = []
    for c in new:
        if c in idx:
            out.append(vals[idx[c]])
            continue
        a = F.covering(idx, *c)
        if a is not None:
            out.append(vals[idx[a]])
        else:
            l, i, j = c
            out.append(np.mean([vals[idx[(l + 1, 2 * i + x, 2 * j + y)]] for x in (0, 1) for y in (0, 1)]))
    return np.array(out)


@pytest.mark.parametrize("kind", [0, 1])
def test_indicator_matches_the_reference(kind):
    wl, F, leaves = vortex_case() if kind == 0 else shore_case()
    ctx = swdg.Context.from_workload(wl)
    ctx.amr_setup(swdg.make_forest(F.nx0, F.ny0, F.x0, F.y0, F.hx0, F.hy0, F.max_level, F.h_min,
                                   F.tags, F.periodic))
    o = Oracle.from_workload(wl)
    ref = indicator(o, wl.mesh, wl.state(), wl.degree, kind, wl.eps_vel)
    got = ctx.amr_indicator(kind)
    assert ref.max() > 0
    np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-12 * ref.max())


def adapt_both(ctx, o, wl, F, leaves, manning, eta, tr, tc):
    """one adaptation of the GPU context and of the reference; returns the new
    leaves, oracle and report"""
    rep = ctx.amr_adapt(tr, tc, eta=eta)
    flags = F.flags(leaves, eta, tr, tc)
    new = F.adapt(leaves, flags)
    np.testing.assert_array_equal(ctx.amr_leaves(), np.array(new, dtype=np.int32))
    state = remap(F, leaves, o.get_state(), new, wl.degree)
    man = carry(F, leaves, new, manning)
    o2 = oracle_of(wl, W.Mesh(*F.mesh(new)), state, man)
    return new, o2, man, rep


def test_one_adaptation_matches_the_reference():
    wl, F, leaves = shore_case(2)
    ctx = swdg.Context.from_workload(wl)
    ctx.amr_setup(swdg.make_forest(F.nx0, F.ny0, F.x0, F.y0, F.hx0, F.hy0, F.max_level, F.h_min,
                                   F.tags, F.periodic))
    o = Oracle.from_workload(wl)
    eta = indicator(o, wl.mesh, wl.state(), wl.degree, 1, wl.eps_vel)
    m0 = o.diagnostics()
    new, o2, man, rep = adapt_both(ctx, o, wl, F, leaves, wl.manning, eta, 0.3, 0.05)
    assert rep["refined"] > 0 and rep["cells_after"] > rep["cells_before"]
    for a, b in zip(ctx.get_state(), o2.get_state()):
        assert rel_inf(a, b, floor=1e-3) <= 1e-12
    # Q^n: the change of the total wet mass across the adaptation
    m1 = o2.diagnostics()
    assert abs(rep["Q"] - (m1["mass"] - m0["mass"])) <= 1e-11 * m0["mass"]
    assert abs(rep["tracer_Q"] - (m1["tracer_mass"] - m0["tracer_mass"])) <= 1e-11 * m0["tracer_mass"]
    # and coarsening back
    eta2 = np.zeros(len(new))
    eta2[0] = 1.0
    new2, o3, _, rep2 = adapt_both(ctx, o2, wl, F, new, man, eta2, 2.0, 0.5)
    assert rep2["coarsened"] > 0
    for a, b in zip(ctx.get_state(), o3.get_state()):
        assert rel_inf(a, b, floor=1e-3) <= 1e-12


@pytest.mark.parametrize("case", ["vortex", "shore"])
def test_adaptive_run_follows_the_oracle_chain(case):
    wl, F, leaves = vortex_case() if case == "vortex" else shore_case()
    kind, tr, tc = (0, 1e-1, 5e-2) if case == "vortex" else (1, 0.3, 0.05)
    ctx = swdg.Context.from_workload(wl)
    ctx.amr_setup(swdg.make_forest(F.nx0, F.ny0, F.x0, F.y0, F.hx0, F.hy0, F.max_level, F.h_min,
                                   F.tags, F.periodic))
    o = Oracle.from_workload(wl)
    man = wl.manning if wl.manning is not None else np.zeros(wl.mesh.n)
    m_start = o.diagnostics()["mass"]
    t = 0.0
    qsum = 0.0
    for cycle in range(3):
        dt = 0.5 * o.cfl_dt(t)  # the step of the current (refined) mesh
        ctx.step(5, dt, t)
        t = o.step(5, dt, t)
        for a, b in zip(ctx.get_state(), o.get_state()):
            assert rel_inf(a, b, floor=1e-3) <= 1e-10
        eta = indicator(o, W.Mesh(*F.mesh(leaves)), o.get_state(), wl.degree, kind, wl.eps_vel)
        leaves, o, man, rep = adapt_both(ctx, o, wl, F, leaves, man, eta, tr, tc)
        qsum += rep["Q"]
    assert len({c[0] for c in leaves}) >= 2
    if case == "vortex":  # flat bottom, all wet, periodic: the remap conserves the mass
        assert abs(o.diagnostics()["mass"] - m_start) <= 1e-12 * m_start
        assert abs(qsum) <= 1e-12 * m_start
