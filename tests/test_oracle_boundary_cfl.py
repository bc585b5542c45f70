"""Pins of the oracle's tidal boundary and of its time step against closed
forms that the scheme fixes.

- Tidal boundary (ghost state of an elevation boundary, R5 reading): on a
  flat bottom of depth D with the interior at rest, the only flux is through
  the tidal faces, where the Rusanov flux of Eq. lxf_parameter with the
  hydrostatic reconstruction of Eq. hydro_rec gives, per unit face length,
  lambda zeta_b / 2 of water (lambda = sqrt(g max(D, D + zeta_b)), the ghost
  elevation zeta_b(t) = A sin(2 pi t / T + phi)) and the non-conservative
  pressure term g (2 D + zeta_b) zeta_b / 4 of x-momentum.  Summing the
  continuity residual over all cells (the test functions sum to one, interior
  fluxes cancel) must give that inflow; over one time step the change of
  water mass must be the tableau's weighted sum of the inflows at the stage
  times t + c_l dt (Sec. 3.1), which a wrong stage time, phase or sign fails.
- Time step of Eq. deltat_fe (Props. 3.2-3.3, R14): for a uniform depth h and
  a uniform stream u in x the per-face-point ratio J_K / (lambda l_Gamma) is
  h_x / (|u| + sqrt(g h)) on x-faces and h_y / sqrt(g h) on y-faces, so on
  rectangular cells dt = C min(h_x / (|u| + c), h_y / c); on a 2:1 forest at
  rest the fine cells bind and a hanging face's coarse side (its J over the
  fine length: twice its width) never does.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle, tableau
from paper_2505_18743_gb300 import workloads as W

G = 9.81


def flat_box(nx, ny, Lx, Ly, depth, degree, pix=2, tags=(0, 0, 0, 0)):
    mesh = W.uniform_mesh(nx, ny, Lx, Ly, tags=tags)
    z = np.full((ny * pix, nx * pix), depth)
    return mesh, W.Raster(z, 0.0, 0.0, Lx / (nx * pix), Ly / (ny * pix))


def tidal_box(degree, mode, D=10.0, amp=0.5, period=3600.0, phase=0.3, **kw):
    mesh, ras = flat_box(6, 4, 600.0, 400.0, D, degree, tags=(1, 0, 0, 0))
    o = Oracle(mesh, ras, degree=degree, subgrid_mode=mode, eps_vel=0.01, h_lim=0.01, **kw)
    o.set_boundary(1, W.BC_TIDE, amp, period, phase)
    nd = (degree + 1) ** 2
    zero = np.zeros((mesh.n, nd))
    o.set_state(zero, zero, zero, np.ones((mesh.n, nd)))
    return o, mesh


def inflow(t, D, amp, period, phase, edge):
    """closed-form water inflow through a tidal edge of length ``edge`` into
    a still flat basin of depth D"""
    zb = amp * np.sin(2 * np.pi * t / period + phase)
    lam = np.sqrt(G * max(D, D + zb))
    return edge * lam * zb / 2, zb


@pytest.mark.parametrize("degree,mode", [(1, 0), (2, 1), (3, 0)])
def test_tidal_face_flux_closed_form(degree, mode):
    D, amp, period, phase = 10.0, 0.5, 3600.0, 0.3
    o, mesh = tidal_box(degree, mode, D, amp, period, phase)
    west = mesh.nbr[:, 0, 0] < 0
    for t in (0.0, 700.0, 1500.0, 2900.0):
        r = o.residual(t)
        flux, zb = inflow(t, D, amp, period, phase, 400.0)
        assert abs(r["F"].sum() - flux) <= 1e-12 * abs(flux) + 1e-12
        # x-momentum: only the pressure term of the tidal faces
        px = 400.0 * G * (2 * D + zb) * zb / 4
        assert abs(r["Gx"].sum() - px) <= 1e-11 * abs(px) + 1e-12
        # nothing moves in y, nothing away from the tidal edge, and a
        # constant tracer enters with the water
        assert np.abs(r["Gy"]).max() <= 1e-9
        assert np.abs(r["F"][~west]).max() <= 1e-12 * abs(flux) + 1e-12
        assert abs(r["R"].sum() - flux) <= 1e-12 * abs(flux) + 1e-12


@pytest.mark.parametrize("tab", [0, 1])
def test_tidal_mass_balance_over_a_step_uses_the_stage_times(tab):
    """One step of length dt = 1e-4 of the CFL step: the stage states barely
    leave rest (their feedback on the boundary flux is ~1e-4 relative), while
    a tide of period 4 dt changes the inflow by O(1) between stage times."""
    D, amp, phase = 10.0, 0.5, 0.4
    o, mesh = tidal_box(1, 0, D, amp, 1.0, phase, tableau=tab)
    dt = 1e-4 * o.cfl_dt(0.0)
    period = 4 * dt
    o.set_boundary(1, W.BC_TIDE, amp, period, phase)
    tb = tableau(tab)
    t0 = 0.37 * period
    m0 = o.diagnostics()["mass"]
    o.step(1, dt, t0)
    dm = o.diagnostics()["mass"] - m0

    def predicted(times):
        return dt * sum(b * inflow(t, D, amp, period, phase, 400.0)[0] for b, t in zip(tb["b"], times))

    right = predicted(t0 + tb["c"] * dt)
    assert abs(dm - right) <= 2e-3 * abs(right)
    # the readings a plausible mistake would take are far off
    for wrong in (predicted(np.full(tb["s"], t0)),            # every stage at the step start
                  predicted(t0 + tb["c"][::-1] * dt),          # stage times permuted
                  -right):                                     # the ghost elevation's sign
        assert abs(dm - wrong) > 0.1 * abs(right)


@pytest.mark.parametrize("degree,mode", [(1, 0), (2, 1), (3, 0)])
@pytest.mark.parametrize("hx,hy,u", [(50.0, 100.0, 1.5), (120.0, 40.0, 0.8), (80.0, 80.0, 2.0)])
def test_cfl_step_closed_form_rectangular_cells_with_a_stream(degree, mode, hx, hy, u):
    h, cfl = 4.0, 0.08
    mesh, ras = flat_box(5, 4, 5 * hx, 4 * hy, h, degree)
    o = Oracle(mesh, ras, degree=degree, subgrid_mode=mode, cfl=cfl, eps_vel=0.01, h_lim=0.01)
    nd = (degree + 1) ** 2
    one = np.ones((mesh.n, nd))
    o.set_state(0 * one, h * u * one, 0 * one, one)
    c = np.sqrt(G * h)
    expect = cfl * min(hx / (u + c), hy / c)
    assert abs(o.cfl_dt(0.0) - expect) <= 1e-13 * expect


@pytest.mark.parametrize("degree", [1, 2])
def test_cfl_step_closed_form_on_a_2to1_forest(degree):
    Lx, Ly, h, cfl = 3200.0, 1600.0, 6.0, 0.1
    mesh, level = W.forest_mesh(8, 4, Lx, Ly, 3, lambda l, x, y, hx, hy: np.abs(x - 1700.0) < 500.0)
    assert (mesh.nbr[:, :, 1] >= 0).sum() > 0 and level.max() == 2
    pix = 16
    z = np.full((4 * pix, 8 * pix), h)
    ras = W.Raster(z, 0.0, 0.0, Lx / (8 * pix), Ly / (4 * pix))
    o = Oracle(mesh, ras, degree=degree, cfl=cfl, eps_vel=0.01, h_lim=0.01)
    nd = (degree + 1) ** 2
    one = np.ones((mesh.n, nd))
    c = np.sqrt(G * h)
    o.set_state(0 * one, 0 * one, 0 * one, one)
    expect = cfl * mesh.hxhy.min() / c
    assert abs(o.cfl_dt(0.0) - expect) <= 1e-13 * expect
    # a stream along x: the fine cells' x-faces bind at h_x / (|u| + c)
    u = 1.2
    o.set_state(0 * one, h * u * one, 0 * one, one)
    fine = level == level.max()
    hxf, hyf = mesh.hxhy[fine, 0].min(), mesh.hxhy[fine, 1].min()
    expect = cfl * min(hxf / (u + c), hyf / c, mesh.hxhy[:, 0].min() / (u + c))
    assert abs(o.cfl_dt(0.0) - expect) <= 1e-13 * expect
