"""Pins of the oracle on 2:1 non-conforming (hanging-face) forests: the
travelling vortex converges at design order across refinement interfaces
that cut through it (Sec. 4.4 on a static refined mesh), the lake at rest is
preserved (Prop. 3.1), free stream is preserved, and mass, tracer mass and
positivity hold across refinement levels (Sec. 3.5)."""
import numpy as np
import pytest

from helpers import Vortex, cell_quadrature
from oracle.oracle import Oracle
from paper_2505_18743_gb300 import workloads as W


def small_lagoon(degree=1, levels=3):
    # a scaled-down lagoon: 32 x 16 coarse cells, 8 px per coarse cell
    return W.lagoon(nx0=32, ny0=16, pix0=8, degree=degree, levels=levels,
                    band=(5000.0, 2500.0))


def hanging_faces(mesh):
    return int((mesh.nbr[:, :, 1] >= 0).sum())


def vortex_forest_error(N, degree, tableau, cfl, band=0.12):
    v = Vortex()
    mesh, level = W.forest_mesh(2 * N, N, v.Lx, v.Ly, 2,
                                lambda l, x, y, hx, hy: np.abs(y - 0.5) < band,
                                periodic=(True, True))
    assert hanging_faces(mesh) > 0
    ras = W.Raster(np.full((N * 8, 2 * N * 8), v.h0), 0.0, 0.0, v.Lx / (2 * N * 8), v.Ly / (N * 8))
    X, Y = W.nodal_coordinates(mesh, degree)
    h, u, w = v(X, Y, 0.0)
    o = Oracle(mesh, ras, degree=degree, tableau=tableau, cfl=cfl, eps_vel=1e-3, h_lim=1e-3)
    o.set_state(h - v.h0, h * u, h * w, np.ones_like(h))
    nst = int(np.ceil(v.T / o.cfl_dt()))
    o.step(nst, v.T / nst)
    px, py, wt = cell_quadrature(mesh, 6)
    z = o.gauges(np.stack([px, py], 1))
    he, _, _ = v(px, py, v.T)
    return float(np.sqrt(np.sum(wt * (z - (he - v.h0)) ** 2)))


def test_vortex_converges_at_design_order_across_hanging_faces():
    e10 = vortex_forest_error(10, 1, 0, 0.25)
    e20 = vortex_forest_error(20, 1, 0, 0.25)
    assert np.log2(e10 / e20) > 1.8
    # between the uniform coarse (N=20: 3.6e-3) and uniform fine (N=40: 8.3e-4) errors
    assert 8.0e-4 < e20 < 3.6e-3


def test_forest_builder_is_2to1_balanced_and_mutual():
    wl = small_lagoon()
    m = wl.mesh
    lev = wl.level
    assert len(np.unique(lev)) == 3 and hanging_faces(m) > 0
    for k in range(m.n):
        for f in range(4):
            s0, s1 = m.nbr[k, f]
            if s0 < 0:
                continue
            for nb in ([s0, s1] if s1 >= 0 else [s0]):
                assert abs(lev[nb] - lev[k]) <= 1
                back = m.nbr[nb, f ^ 1]
                assert k in back


@pytest.mark.parametrize("degree", [1, 2])
def test_lake_at_rest_on_forest(degree):
    wl = small_lagoon(degree)
    wl.boundaries = []  # walls everywhere: no tide
    o = Oracle.from_workload(wl)
    z = o.lake_at_rest(0.0)
    zero = np.zeros_like(z)
    o.set_state(z, zero, zero, np.ones_like(z))
    r = o.residual(0.0)
    for k, v in r.items():
        assert np.abs(v).max() < 1e-9, k  # O(1e-13) relative to the O(1e4) face terms
    o.step(10, -1.0, 0.0)
    z1, qx, qy, c = o.get_state()
    assert np.abs(z1 - z).max() < 1e-13
    assert np.abs(qx).max() < 1e-13 and np.abs(qy).max() < 1e-13


def test_free_stream_on_forest():
    mesh, _ = W.forest_mesh(6, 4, 60.0, 40.0, 3, lambda l, x, y, hx, hy: (x > 20) & (x < 45),
                            periodic=(True, True))
    assert hanging_faces(mesh) > 0
    ras = W.Raster(np.full((32, 48), 3.0), 0.0, 0.0, 60.0 / 48, 40.0 / 32)
    for degree in (1, 2, 3):
        o = Oracle(mesh, ras, degree=degree)
        one = np.ones((mesh.n, (degree + 1) ** 2))
        o.set_state(0.25 * one, 1.3 * one, -0.7 * one, 0.4 * one)
        for k, v in o.residual().items():
            assert np.abs(v).max() < 1e-12, (degree, k)


def test_mass_tracer_positivity_across_levels():
    wl = small_lagoon(1)
    wl.boundaries = []  # closed basin
    Xn, Yn = W.nodal_coordinates(wl.mesh, 1)
    wl.zeta = 0.8 * np.exp(-((Xn - 15000.0) ** 2 + (Yn - 12000.0) ** 2) / 3000.0 ** 2)
    wl.c = np.ones_like(wl.zeta)
    o = Oracle.from_workload(wl, newton_max=3)
    d0 = o.diagnostics()
    for _ in range(20):
        o.step(1)
    d1 = o.diagnostics()
    assert d1["r_cells"] < wl.mesh.n  # wet-dry cells present
    assert abs(d1["mass"] - d0["mass"]) <= 1e-13 * d0["mass"]
    assert abs(d1["tracer_mass"] - d0["tracer_mass"]) <= 1e-13 * d0["tracer_mass"]
    assert d1["positivity_violations"] == 0
    assert np.abs(o.get_state()[3] - 1.0).max() < 1e-12
