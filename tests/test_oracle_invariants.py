"""Pins of the whole oracle against the properties the paper proves or
measures: well-balancing (Prop. 3.1, Table tab:lake_at_rest_pert_rest), mass
conservation (Sec. 3.5), positivity under the CFL bound (Props. 3.2-3.3),
consistency with continuity (Eq. cwc1), Newton convergence (Sec. 3.4) and
free-stream preservation of the DG operator."""
import numpy as np
import pytest

from helpers import golden_rows
from oracle.oracle import Oracle
from paper_2505_18743_gb300 import workloads as W


def lake(degree, submerged, n=8, pix=4, mode=0, tableau=0):
    wl = W.lake_at_rest_bump(n=n, pix=pix, degree=degree, submerged=submerged)
    wl.subgrid_mode = mode
    wl.tableau = tableau
    o = Oracle.from_workload(wl)
    z = o.lake_at_rest(0.0)
    zero = np.zeros_like(z)
    o.set_state(z, zero, zero, np.ones_like(z))
    return wl, o


def l2(mesh, a):
    J = mesh.hxhy[:, 0] * mesh.hxhy[:, 1]
    return float(np.sqrt(np.sum(J[:, None] * a ** 2) / a.shape[1]))


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("degree", [1, 2, 3])
@pytest.mark.parametrize("submerged", [True, False])
def test_lake_at_rest_is_preserved(degree, submerged, mode):
    """Prop. 3.1 with the paper's bump (discontinuous submerged / emerged
    wet-dry); the errors must stay at the round-off level the paper prints."""
    wl, o = lake(degree, submerged, mode=mode)
    rows = golden_rows("lake_at_rest.txt")
    bound = 5 * max(float(r[2]) for r in rows) + 1e-14  # printed errors are <= 1.5e-13
    res = o.residual()
    for k, v in res.items():
        assert np.abs(v).max() < 1e-13 * 9.81, k
    z0, qx0, qy0, c0 = o.get_state()
    t = o.step(25)
    z, qx, qy, c = o.get_state()
    assert t > 0
    assert l2(wl.mesh, z - z0) <= bound
    assert l2(wl.mesh, qx) <= bound and l2(wl.mesh, qy) <= bound
    assert np.abs(c - 1).max() < 1e-13
    if not submerged:
        assert o.diagnostics()["r_cells"] < wl.mesh.n  # wet-dry cells switched to r_K = 0


def island(degree=1, cfl_scale=0.9, newton_max=20, amp=0.5, tableau=0, mode=0):
    """closed basin with an emerged island and a hump of water next to it"""
    wl = W.closed_basin(degree=degree)
    n = wl.raster.z.shape[0]
    dx = wl.raster.dx
    xc = (np.arange(n) + 0.5) * dx
    X, Y = np.meshgrid(xc, xc)
    wl.raster.z = wl.raster.z - 8.0 * np.exp(-((X - 500) ** 2 + (Y - 500) ** 2) / 150.0 ** 2)
    Xn, Yn = W.nodal_coordinates(wl.mesh, degree)
    wl.zeta = amp * np.exp(-((Xn - 300) ** 2 + (Yn - 500) ** 2) / 100.0 ** 2)
    wl.c = np.ones_like(wl.zeta)
    wl.tableau = tableau
    wl.subgrid_mode = mode
    bound = {1: 1 / 6, 2: 1 / 12, 3: 1 / 20}[degree]
    wl.cfl = cfl_scale * (bound / (2 - np.sqrt(2)) if tableau == 0 else bound)
    return wl, Oracle.from_workload(wl, newton_max=newton_max)


def test_closed_basin_conserves_mass_and_tracer():
    wl = W.closed_basin()
    o = Oracle.from_workload(wl)
    d0 = o.diagnostics()
    o.step(100)
    d1 = o.diagnostics()
    assert abs(d1["mass"] - d0["mass"]) <= 1e-13 * d0["mass"]
    assert abs(d1["tracer_mass"] - d0["tracer_mass"]) <= 1e-13 * d0["tracer_mass"]
    assert d1["newton_max"] == 2  # fully wet: M constant, 2nd iterate converged (Sec. 3.4)
    assert d1["positivity_violations"] == 0


@pytest.mark.parametrize("degree,mode", [(1, 0), (2, 0), (1, 1)])
def test_wet_dry_mass_positivity_and_cwc(degree, mode):
    """Moving wet-dry front around an island: mass and tracer mass to round-off,
    no positivity violation at the RK32 bound (Prop. 3.3), c = 1 preserved
    (Eq. cwc1), and two Newton iterations are enough (Sec. 4.3, Sec. 5)."""
    wl, o = island(degree, newton_max=2, mode=mode)
    d0 = o.diagnostics()
    for _ in range(40):
        o.step(1)
    d1 = o.diagnostics()
    z, qx, qy, c = o.get_state()
    assert d1["r_cells"] < wl.mesh.n
    assert abs(d1["mass"] - d0["mass"]) <= 1e-13 * d0["mass"]
    assert abs(d1["tracer_mass"] - d0["tracer_mass"]) <= 1e-13 * d0["tracer_mass"]
    assert d1["positivity_violations"] == 0
    assert np.abs(c - 1.0).max() < 1e-12
    assert o.cell_mass().min() >= 0.0


def test_positivity_violations_reported_above_the_bound():
    wl, o = island(1, cfl_scale=3.0, amp=2.0)
    for _ in range(30):
        o.step(1)
    assert o.diagnostics()["positivity_violations"] > 0


def test_degree_switch_and_remap_are_mass_exact():
    wl, o = island(2, amp=0.5)
    # make the tracer non-constant so the remap has work to do
    Xn, Yn = W.nodal_coordinates(wl.mesh, 2)
    z, qx, qy, c = o.get_state()
    o.set_state(z, qx + 0.1 * np.sin(Xn / 90.0), qy, 0.5 + 0.4 * np.cos(Yn / 70.0))
    d0 = o.diagnostics()
    o.degree_switch()
    f = o.flags()
    d1 = o.diagnostics()
    z1, qx1, qy1, c1 = o.get_state()
    assert (f == 0).sum() > 0 and (f == 2).sum() > 0
    assert abs(d1["mass"] - d0["mass"]) <= 1e-13 * d0["mass"]
    assert abs(d1["tracer_mass"] - d0["tracer_mass"]) <= 1e-13 * d0["tracer_mass"]
    for fld in (z1, qx1, c1):
        assert np.all(fld[f == 0] == fld[f == 0][:, :1])  # constants on r_K = 0 cells
    np.testing.assert_array_equal(z1[f == 2], z[f == 2])


def test_wall_boundary_and_interior_faces_conserve_mass_exactly_per_step():
    """sum over cells of the continuity residual vanishes in a closed basin
    for any state (interior fluxes cancel, wall flux is zero)"""
    wl = W.closed_basin(degree=2)
    rng = np.random.default_rng(11)
    o = Oracle.from_workload(wl)
    nd = 9
    o.set_state(rng.normal(0, 0.2, (wl.mesh.n, nd)), rng.normal(0, 1, (wl.mesh.n, nd)),
                rng.normal(0, 1, (wl.mesh.n, nd)), rng.uniform(0, 1, (wl.mesh.n, nd)))
    r = o.residual()
    assert abs(r["F"].sum()) < 1e-10 * np.abs(r["F"]).sum()
    assert abs(r["R"].sum()) < 1e-10 * np.abs(r["R"]).sum()


@pytest.mark.parametrize("degree", [1, 2, 3])
def test_free_stream_preservation(degree):
    """a uniform flow over a flat bed in a periodic box has zero residual:
    volume and face terms of every equation cancel exactly (up to round-off)"""
    mesh, ras = W.flat_periodic(5, 4, 50.0, 40.0, 3.0, degree, pix=2)
    o = Oracle(mesh, ras, degree=degree)
    nd = (degree + 1) ** 2
    one = np.ones((mesh.n, nd))
    o.set_state(0.25 * one, 1.3 * one, -0.7 * one, 0.4 * one)
    r = o.residual()
    for k, v in r.items():
        assert np.abs(v).max() < 1e-12, k


def test_dry_cells_stay_dry_and_untouched():
    wl, o = lake(2, submerged=False, n=16)
    z0 = o.get_state()[0]
    f0 = o.flags()
    o.step(5)
    z1 = o.get_state()[0]
    dry = np.all(z0 == z0[:, :1], axis=1) & (z0[:, 0] != 0.0)  # Def. 3.1 dry level
    assert dry.sum() > 0
    np.testing.assert_array_equal(z1[dry], z0[dry])
    assert f0.shape[0] == wl.mesh.n
