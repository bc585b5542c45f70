"""Parity of the CUDA path (through the C-ABI) with the FP64 CPU oracle.

Tolerances: residuals within 1e-12 relative per field (max abs difference over
the field's own max |oracle|; lake-at-rest cases, whose residuals are round-off,
use absolute bounds instead); states within 1e-10 relative per field after the
stated number of steps (elevation and tracer against max(|oracle|, 1),
discharges against max(|oracle|, 1e-3)); integer decisions (degree flags)
bit-exact.
"""
import numpy as np
import pytest

from helpers import rel_inf, residual_errors
from oracle.oracle import Oracle
from paper_2505_18743_gb300 import swdg
from paper_2505_18743_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RES_TOL = 1e-12
STATE_TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _build():
    import torch
    assert torch.cuda.is_available()
    from paper_2505_18743_gb300 import build as B
    from oracle import oracle
    B.build()
    oracle.build()


def pair(wl, **over):
    return swdg.Context.from_workload(wl, **over), Oracle.from_workload(wl, **over)


def check_residual(ctx, ora, t=0.0, tol=RES_TOL):
    rg = ctx.residual(t)
    ro = ora.residual(t)
    worst = residual_errors(rg, ro)
    for k, err in worst.items():
        assert err <= tol, (k, err, worst)
    return worst


def check_state(ctx, ora, tol=STATE_TOL):
    sg, so = ctx.get_state(), ora.get_state()
    errs = []
    for name, a, b in zip(("zeta", "qx", "qy", "c"), sg, so):
        floor = 1.0 if name in ("zeta", "c") else 1e-3
        e = rel_inf(a, b, floor=floor)
        errs.append(e)
        assert e <= tol, (name, e)
    return errs


def randomize(wl, seed=3, amp_q=0.5, amp_z=0.05):
    rng = np.random.default_rng(seed)
    sh = wl.zeta.shape
    wl.zeta = wl.zeta + amp_z * rng.standard_normal(sh)
    wl.qx = amp_q * rng.standard_normal(sh)
    wl.qy = amp_q * rng.standard_normal(sh)
    wl.c = rng.uniform(0, 1, sh)
    return wl


def island(degree=1, amp=0.5, tableau=0, mode=0, n=16):
    wl = W.closed_basin(degree=degree, n=n)
    npx = wl.raster.z.shape[0]
    xc = (np.arange(npx) + 0.5) * wl.raster.dx
    X, Y = np.meshgrid(xc, xc)
    wl.raster.z = wl.raster.z - 8.0 * np.exp(-((X - 500) ** 2 + (Y - 500) ** 2) / 150.0 ** 2)
    Xn, Yn = W.nodal_coordinates(wl.mesh, degree)
    wl.zeta = amp * np.exp(-((Xn - 300) ** 2 + (Yn - 500) ** 2) / 100.0 ** 2)
    wl.c = 0.5 + 0.4 * np.cos(Yn / 70.0)
    wl.tableau = tableau
    wl.subgrid_mode = mode
    b = {1: 1 / 6, 2: 1 / 12, 3: 1 / 20}[degree]
    wl.cfl = 0.9 * (b / (2 - np.sqrt(2)) if tableau == 0 else b)
    return wl


# ----------------------------------------------------------------------------
# residual
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("degree", [1, 2, 3])
def test_residual_closed_basin_random_state(degree, mode):
    wl = randomize(W.closed_basin(degree=degree))
    wl.subgrid_mode = mode
    ctx, ora = pair(wl)
    check_residual(ctx, ora)


def test_residual_closed_basin_paper_config():
    wl = W.closed_basin()
    ctx, ora = pair(wl)
    check_residual(ctx, ora)


@pytest.mark.parametrize("degree", [1, 2, 3])
def test_residual_wet_dry_island_with_friction(degree):
    wl = island(degree, amp=1.5)
    wl.manning = np.full(wl.mesh.n, 0.03)
    wl.qx = 0.3 * np.ones_like(wl.zeta)
    ctx, ora = pair(wl)
    check_residual(ctx, ora)


def test_residual_tidal_beach_crops_float32_raster():
    # west-boundary crop (tide) and a shoreline crop (wet-dry, east wall)
    for window, t in [((0, 100, 8, 8), 3000.0), ((236, 120, 20, 12), 0.0)]:
        wl = W.tidal_beach(window=window)
        Xn, Yn = W.nodal_coordinates(wl.mesh, 3)
        wl.zeta = 0.3 * np.sin(Xn / 400.0) * np.cos(Yn / 300.0)
        wl.qx = 0.2 * np.cos(Yn / 200.0) * np.ones_like(Xn)
        ctx, ora = pair(wl)
        assert wl.raster.z.dtype == np.float32
        check_residual(ctx, ora, t)


# ----------------------------------------------------------------------------
# time step, degree switch, diagnostics, gauges
# ----------------------------------------------------------------------------
def test_cfl_dt_matches():
    for wl in (randomize(W.closed_basin(degree=2)), island(2)):
        ctx, ora = pair(wl)
        dg, do = ctx.cfl_dt(0.0), ora.cfl_dt(0.0)
        assert abs(dg - do) <= 1e-13 * do


@pytest.mark.parametrize("degree", [1, 2, 3])
def test_degree_switch_flags_bitexact_and_remap(degree):
    wl = island(degree, amp=0.5)
    Xn, Yn = W.nodal_coordinates(wl.mesh, degree)
    wl.qx = 0.1 * np.sin(Xn / 90.0)
    ctx, ora = pair(wl)
    fg = ctx.degree_switch()
    ora.degree_switch()
    fo = ora.flags()
    np.testing.assert_array_equal(fg, fo)
    assert (fo == 0).sum() > 0
    check_state(ctx, ora, tol=1e-12)


def test_diagnostics_and_gauges_match():
    wl = island(2, amp=0.5)
    ctx, ora = pair(wl)
    dg, do = ctx.diagnostics(), ora.diagnostics()
    for k in ("mass", "tracer_mass"):
        assert abs(dg[k] - do[k]) <= 1e-13 * do[k], k
    assert abs(dg["min_h"] - do["min_h"]) <= 1e-12
    rng = np.random.default_rng(5)
    xy = rng.uniform(1.0, 999.0, size=(50, 2))
    zg, zo = ctx.gather_gauges(xy), ora.gauges(xy)
    assert np.abs(zg - zo).max() <= 1e-13


def test_closed_basin_100_ssp33_steps():
    """the paper-scale closed basin: 100 SSP33 steps at CFL 0.1"""
    wl = W.closed_basin()
    ctx, ora = pair(wl)
    tg = ctx.step(100, -1.0, 0.0)
    to = ora.step(100, -1.0, 0.0)
    assert abs(tg - to) <= 1e-10 * to
    check_state(ctx, ora)
    dg, do = ctx.diagnostics(), ora.diagnostics()
    # fully wet: the oracle verifies the first iterate with a second Newton step
    # (Sec. 3.4); the CUDA path certifies it instead (affine H, exact Jacobian)
    assert do["newton_max"] == 2 and dg["newton_max"] == 1


@pytest.mark.parametrize("degree,mode", [(1, 0), (2, 0), (1, 1), (3, 0)])
def test_wet_dry_island_steps(degree, mode):
    wl = island(degree, amp=0.5, mode=mode, n=12 if degree == 3 else 16)
    ctx, ora = pair(wl)
    d0 = ctx.diagnostics()
    tg = ctx.step(20, -1.0, 0.0)
    to = ora.step(20, -1.0, 0.0)
    assert abs(tg - to) <= 1e-10 * to
    check_state(ctx, ora)
    d1 = ctx.diagnostics()
    assert abs(d1["mass"] - d0["mass"]) <= 1e-13 * d0["mass"]
    assert d1["positivity_violations"] == 0
    assert d1["r_cells"] == ora.diagnostics()["r_cells"]


def test_tidal_beach_crop_rk32_imex_with_friction():
    wl = W.tidal_beach(window=(0, 120, 12, 8))
    wl.zeta = 0.2 * np.ones_like(wl.zeta)
    ctx, ora = pair(wl)
    tg = ctx.step(20, -1.0, 1000.0)
    to = ora.step(20, -1.0, 1000.0)
    assert abs(tg - to) <= 1e-10 * to
    check_state(ctx, ora)


def test_shoreline_crop_rk32_wet_dry():
    wl = W.tidal_beach(window=(236, 120, 16, 8))
    Xn, Yn = W.nodal_coordinates(wl.mesh, 3)
    wl.zeta = 0.5 * np.exp(-((Xn - 18900.0) / 200.0) ** 2)
    ctx, ora = pair(wl)
    ctx.step(10, -1.0, 0.0)
    ora.step(10, -1.0, 0.0)
    check_state(ctx, ora)


def _steps_with_diagnostics(ctx, ora, n, t0):
    d0 = ctx.diagnostics()
    tg = ctx.step(n, -1.0, t0)
    to = ora.step(n, -1.0, t0)
    assert abs(tg - to) <= 1e-10 * to
    errs = check_state(ctx, ora)
    dg, do = ctx.diagnostics(), ora.diagnostics()
    assert dg["positivity_violations"] == 0 and do["positivity_violations"] == 0
    assert dg["r_cells"] == do["r_cells"]
    for k in ("mass", "tracer_mass"):
        assert abs(dg[k] - do[k]) <= 1e-12 * do[k], k
    return d0, dg, errs


def test_tidal_west_crop_64x64_r3_100_rk32_steps():
    """100 RK32-IMEX steps of a 64 x 64-cell crop of the 256 x 256, r = 3
    tidal beach that carries the tidal west boundary: the run starts at
    t = 3000 s, when the boundary elevation is 0.41 m above the still
    interior, so a bore enters through the tidal faces; with friction and a
    moving offshore hump.  States within 1e-10 of the oracle."""
    wl = W.tidal_beach(window=(0, 96, 64, 64))
    Xn, Yn = W.nodal_coordinates(wl.mesh, 3)
    wl.zeta = 0.3 * np.exp(-((Xn - 3000.0) ** 2 + (Yn - 10000.0) ** 2) / 600.0 ** 2)
    wl.qx = 0.5 * np.cos(Yn / 700.0)
    wl.qy = 0.2 * np.sin(Xn / 900.0)
    ctx, ora = pair(wl)
    _steps_with_diagnostics(ctx, ora, 100, 3000.0)


def test_shoreline_crop_64x64_r3_100_rk32_steps():
    """100 RK32-IMEX steps of the 64 x 64-cell crop of the beach that holds
    the shoreline band (x = 15..20 km, the linear slope from 30 m depth to
    5 m above datum with the under-resolved channels): a 0.8 m wave runs up
    the beach, so wet-dry fronts move through the pixel tiles, cells switch
    degree and the Newton solves take their masked and dry paths.  States
    within 1e-10 of the oracle."""
    wl = W.tidal_beach(window=(192, 96, 64, 64))
    Xn, Yn = W.nodal_coordinates(wl.mesh, 3)
    wl.zeta = 0.8 * np.exp(-((Xn - 18700.0) / 300.0) ** 2) * (1.0 + 0.3 * np.cos(Yn / 500.0))
    # a discharge only offshore: q = 0 where the land is dry
    wl.qx = np.where(Xn < 18500.0, 0.4 * np.exp(-((Xn - 18000.0) / 500.0) ** 2), 0.0)
    ctx, ora = pair(wl)
    d0, d1, _ = _steps_with_diagnostics(ctx, ora, 100, 0.0)
    # the walls close this crop: water mass is conserved to round-off
    assert abs(d1["mass"] - d0["mass"]) <= 1e-13 * d0["mass"]
    assert 0 < d1["r_cells"] < wl.mesh.n


@pytest.mark.slow
def test_full_size_tidal_beach_10_rk32_steps():
    """the whole 256 x 256, r = 3, 16 x 16 px/cell tidal beach for 10
    RK32-IMEX steps from t = 3000 s (tide entering at the west, a disturbed
    interior, the shoreline in the east), every cell against the oracle."""
    wl = W.tidal_beach()
    Xn, Yn = W.nodal_coordinates(wl.mesh, 3)
    wl.zeta = 0.4 * np.sin(Xn / 700.0) * np.cos(Yn / 500.0)
    wl.qx = np.where(Xn < 18500.0, 0.3 * np.cos(Yn / 900.0), 0.0)  # none on dry land
    ctx, ora = pair(wl)
    _steps_with_diagnostics(ctx, ora, 10, 3000.0)


@pytest.mark.parametrize("tableau", [2, 3])
def test_other_tableaux(tableau):
    wl = randomize(W.closed_basin(degree=2), amp_q=0.05, amp_z=0.01)
    wl.tableau = tableau
    wl.cfl = 0.05
    ctx, ora = pair(wl)
    ctx.step(5, -1.0, 0.0)
    ora.step(5, -1.0, 0.0)
    check_state(ctx, ora)


# ----------------------------------------------------------------------------
# invariants on the GPU path itself
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("degree", [1, 2, 3])
def test_gpu_lake_at_rest_well_balanced(degree):
    wl = W.lake_at_rest_bump(n=8, pix=4, degree=degree, submerged=False)
    ora = Oracle.from_workload(wl)
    z = ora.lake_at_rest(0.0)
    zero = np.zeros_like(z)
    wl.zeta, wl.qx, wl.qy, wl.c = z, zero, zero.copy(), np.ones_like(z)
    ctx = swdg.Context.from_workload(wl)
    r = ctx.residual(0.0)
    for k, v in r.items():
        assert np.abs(v).max() < 1e-13 * 9.81, k
    ctx.step(25, -1.0, 0.0)
    zg, qxg, qyg, cg = ctx.get_state()
    assert np.abs(zg - z).max() < 1e-13
    assert np.abs(qxg).max() < 1e-13 and np.abs(qyg).max() < 1e-13
    assert np.abs(cg - 1).max() < 1e-13


def test_gpu_mass_conservation_closed_basin_wet_dry():
    wl = island(2, amp=1.0)
    ctx = swdg.Context.from_workload(wl)
    d0 = ctx.diagnostics()
    ctx.step(100, -1.0, 0.0)
    d1 = ctx.diagnostics()
    assert abs(d1["mass"] - d0["mass"]) <= 1e-13 * d0["mass"]
    assert abs(d1["tracer_mass"] - d0["tracer_mass"]) <= 1e-13 * d0["tracer_mass"]


def test_full_size_tidal_beach_sampled_residual():
    """the 256 x 256, r = 3, 16 x 16 px/cell workload at full size: the oracle
    evaluates a sample of cells one by one"""
    wl = W.tidal_beach()
    Xn, Yn = W.nodal_coordinates(wl.mesh, 3)
    wl.zeta = 0.4 * np.sin(Xn / 700.0) * np.cos(Yn / 500.0)
    wl.qx = 0.3 * np.cos(Yn / 900.0)
    ctx = swdg.Context.from_workload(wl)
    ora = Oracle.from_workload(wl)
    rg = ctx.residual(2000.0)
    rng = np.random.default_rng(8)
    cells = np.concatenate([rng.choice(wl.mesh.n, 200, replace=False),
                            np.arange(0, wl.mesh.n, 256)[:50],              # west boundary (tide)
                            np.arange(250, wl.mesh.n, 256)[::5]])           # shoreline
    ro = ora.residual(2000.0, cells=cells)
    errs = residual_errors({k: v[cells] for k, v in rg.items()}, ro)
    assert max(errs.values()) <= RES_TOL, errs


# ----------------------------------------------------------------------------
# 2:1 non-conforming forests (hanging faces), pixel counts 32/16/8 per level
# ----------------------------------------------------------------------------
def small_lagoon(degree=1, levels=3):
    return W.lagoon(nx0=32, ny0=16, pix0=8, degree=degree, levels=levels,
                    band=(5000.0, 2500.0))


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("degree", [1, 2, 3])
def test_residual_forest_random_state(degree, mode):
    wl = randomize(small_lagoon(degree), amp_q=0.3, amp_z=0.2)
    wl.subgrid_mode = mode
    assert (wl.mesh.nbr[:, :, 1] >= 0).sum() > 0
    ctx, ora = pair(wl)
    check_residual(ctx, ora, 3000.0)


def test_forest_lake_at_rest_and_steps():
    wl = small_lagoon(2)
    wl.boundaries = []
    ora = Oracle.from_workload(wl)
    z = ora.lake_at_rest(0.0)
    zero = np.zeros_like(z)
    wl.zeta, wl.qx, wl.qy, wl.c = z, zero, zero.copy(), np.ones_like(z)
    ctx = swdg.Context.from_workload(wl)
    for k, v in ctx.residual(0.0).items():
        assert np.abs(v).max() < 1e-9, k
    ctx.step(10, -1.0, 0.0)
    zg, qxg, qyg, _ = ctx.get_state()
    assert np.abs(zg - z).max() < 1e-13 and np.abs(qxg).max() < 1e-13


@pytest.mark.parametrize("degree", [1, 2])
def test_forest_tidal_steps(degree):
    wl = small_lagoon(degree)
    Xn, Yn = W.nodal_coordinates(wl.mesh, degree)
    wl.zeta = 0.3 * np.exp(-((Xn - 20000.0) ** 2 + (Yn - 12000.0) ** 2) / 4000.0 ** 2)
    ctx, ora = pair(wl)
    d0 = ctx.diagnostics()
    tg = ctx.step(15, -1.0, 2000.0)
    to = ora.step(15, -1.0, 2000.0)
    assert abs(tg - to) <= 1e-10 * to
    check_state(ctx, ora)
    assert ctx.diagnostics()["positivity_violations"] == 0


def test_forest_vortex_steps_match():
    from helpers import Vortex
    v = Vortex()
    N = 10
    mesh, _ = W.forest_mesh(2 * N, N, v.Lx, v.Ly, 2, lambda l, x, y, hx, hy: np.abs(y - 0.5) < 0.12,
                            periodic=(True, True))
    ras = W.Raster(np.full((N * 8, 2 * N * 8), v.h0), 0.0, 0.0, v.Lx / (2 * N * 8), v.Ly / (N * 8))
    X, Y = W.nodal_coordinates(mesh, 2)
    h, u, w = v(X, Y, 0.0)
    wl = W.Workload("vortex-forest", 2, mesh, ras, h - v.h0, h * u, h * w, np.ones_like(h),
                    tableau=1, cfl=0.1, eps_vel=1e-3, h_lim=1e-3)
    ctx, ora = pair(wl)
    ctx.step(30, -1.0, 0.0)
    ora.step(30, -1.0, 0.0)
    check_state(ctx, ora)


def test_full_size_lagoon_sampled_residual():
    """the 50 km x 30 km lagoon forest (about 200k cells, r = 2) at full size:
    the oracle evaluates a sample of cells one by one, hanging ones included"""
    wl = W.lagoon()
    Xn, Yn = W.nodal_coordinates(wl.mesh, 2)
    wl.zeta = 0.4 * np.sin(Xn / 3000.0) * np.cos(Yn / 2000.0)
    wl.qx = 0.2 * np.cos(Yn / 4000.0)
    ctx = swdg.Context.from_workload(wl)
    ora = Oracle.from_workload(wl)
    rg = ctx.residual(5000.0)
    rng = np.random.default_rng(9)
    hang = np.where((wl.mesh.nbr[:, :, 1] >= 0).any(axis=1))[0]
    fine = np.where((wl.level == 2))[0]
    cells = np.unique(np.concatenate([rng.choice(wl.mesh.n, 150, replace=False),
                                      rng.choice(hang, 100, replace=False),
                                      rng.choice(fine, 50, replace=False)]))
    ro = ora.residual(5000.0, cells=cells)
    errs = residual_errors({k: v[cells] for k, v in rg.items()}, ro)
    assert max(errs.values()) <= RES_TOL, errs


# ----------------------------------------------------------------------------
# errors are reported, never trapped
# ----------------------------------------------------------------------------
def test_errors_are_reported():
    wl = W.closed_basin()
    ctx = swdg.Context(**wl.config())
    with pytest.raises(swdg.SwdgError) as e:
        ctx.set_state(*wl.state())
    assert e.value.code == swdg.SWDG_ESTATE
    bad = wl.mesh.nbr.copy()
    bad[3, 1, 1] = 5  # a 2:1 face whose fine cells do not fit the coarse face
    with pytest.raises(swdg.SwdgError) as e:
        ctx.upload_mesh(wl.mesh.x0y0, wl.mesh.hxhy, bad)
    assert e.value.code == swdg.SWDG_EINVAL
    ctx.upload_mesh(wl.mesh.x0y0, wl.mesh.hxhy, wl.mesh.nbr)
    with pytest.raises(swdg.SwdgError) as e:  # pixels not aligned with the cells
        ctx.upload_bathymetry(wl.raster.z, 1.3, 0.0, wl.raster.dx, wl.raster.dy)
    assert e.value.code == swdg.SWDG_EINVAL
    ctx.upload_bathymetry(wl.raster.z, 0.0, 0.0, wl.raster.dx, wl.raster.dy)
    ctx.set_state(*wl.state())
    # a NaN elevation reads as dry (every wet/dry comparison is false) and is
    # absorbed; a NaN discharge propagates through the fluxes and is reported
    qx = wl.qx.copy()
    qx[7, 0] = np.nan
    ctx.set_state(wl.zeta, qx, wl.qy, wl.c)
    with pytest.raises(swdg.SwdgError) as e:
        ctx.step(1, -1.0, 0.0)
    assert e.value.code == swdg.SWDG_ENAN


@pytest.mark.parametrize("degree", [1, 2, 3])
def test_residual_and_steps_with_tracer_diffusion(degree):
    # Eq. numdiff with a per-cell diffusivity, on the shoreline crop (wet, dry, partly wet)
    wl = W.tidal_beach(window=(232, 118, 8, 6), degree=degree, pix=16)
    Xn, Yn = W.nodal_coordinates(wl.mesh, degree)
    wl.zeta = 0.2 + 0.1 * np.sin(Xn / 300.0) * np.cos(Yn / 250.0)  # every field carries signal
    wl.qx = 0.1 * np.cos(Yn / 200.0) + 0.0 * Xn
    wl.qy = 0.05 * np.sin(Xn / 170.0)
    wl.c = 0.5 + 0.4 * np.sin(Xn / 150.0) * np.cos(Yn / 120.0)
    wl.tracer_diffusivity = np.linspace(0.5, 4.0, wl.mesh.n)
    ctx, ora = pair(wl)
    check_residual(ctx, ora, t=500.0)
    ctx.step(6, -1.0, 0.0)
    ora.step(6, -1.0, 0.0)
    check_state(ctx, ora)
    # without diffusion the tracer differs: the term is active
    plain, _ = pair(W.tidal_beach(window=(232, 118, 8, 6), degree=degree, pix=16))
    plain.set_state(*wl.state())
    plain.step(6, -1.0, 0.0)
    assert np.abs(plain.get_state()[3] - ctx.get_state()[3]).max() > 1e-8


def test_thacker_paraboloid_steps_mode_p():
    """Thacker's oscillating paraboloid (Sec. 4.3) in the sampling mode of the
    paper (mode P), r = 1 on 25 x 25 cells: 60 RK32-IMEX steps (0.8 of an
    oscillation period: the shoreline moves through the cells, which switch
    degree) against the oracle; states within 1e-10, water and tracer mass
    kept."""
    from helpers import Thacker
    th = Thacker()
    N, pix = 25, 4
    mesh = W.uniform_mesh(N, N, th.L, th.L)
    npx = N * pix
    dx = th.L / npx
    xc = (np.arange(npx) + 0.5) * dx
    Xp, Yp = np.meshgrid(xc, xc)
    ras = W.Raster(th.zb(Xp, Yp), 0.0, 0.0, dx, dx)
    X, Y = W.nodal_coordinates(mesh, 1)
    z, u, v = th(X, Y, 0.0)
    b = th.zb(X, Y)
    h = np.maximum(z + b, 0.0)
    z = np.where(h > 0, z, -b)
    wl = W.Workload("thacker-25", 1, mesh, ras, z, h * u, h * v, np.ones_like(z), tableau=0,
                    cfl=0.9 * 0.28, eps_vel=th.eps400 * 400 / N, h_lim=th.h_lim, subgrid_mode=1)
    ctx, ora = pair(wl)
    d0 = ctx.diagnostics()
    _, d1, _ = _steps_with_diagnostics(ctx, ora, 60, 0.0)
    assert abs(d1["mass"] - d0["mass"]) <= 1e-13 * d0["mass"]
    assert abs(d1["tracer_mass"] - d0["tracer_mass"]) <= 1e-13 * d0["tracer_mass"]
    assert 0 < d1["r_cells"] < wl.mesh.n


# ----------------------------------------------------------------------------
# degenerate cases
# ----------------------------------------------------------------------------
def one_cell(degree, mode):
    """a single 100 m cell with walls on all four faces, a 3 m bump under 5 m
    of water (16 x 16 pixels), a tilted surface, discharges and a tracer
    gradient"""
    L, P = 100.0, 16
    mesh = W.uniform_mesh(1, 1, L, L)
    dx = L / P
    xc = (np.arange(P) + 0.5) * dx
    Xp, Yp = np.meshgrid(xc, xc)
    ras = W.Raster(5.0 - 3.0 * np.exp(-((Xp - 60) ** 2 + (Yp - 40) ** 2) / 30.0 ** 2), 0.0, 0.0, dx, dx)
    X, Y = W.nodal_coordinates(mesh, degree)
    zeta = 0.3 * (X - 50) / 50
    qx = 0.2 * np.sin(np.pi * X / L)
    qy = -0.1 * np.sin(np.pi * Y / L)
    c = 0.5 + 0.3 * X / L
    b = {1: 1 / 6, 2: 1 / 12, 3: 1 / 20}[degree]
    return W.Workload("one-cell", degree, mesh, ras, zeta, qx, qy, c, tableau=0,
                      cfl=0.9 * b / (2 - np.sqrt(2)), subgrid_mode=mode)


@pytest.mark.parametrize("mode", [0, 1])
def test_single_cell_domain(mode):
    """one cell (an odd count: the stage update's second team has no cell),
    walls only: residual and 30 RK32-IMEX steps against the oracle"""
    wl = one_cell(3, mode)
    ctx, ora = pair(wl)
    check_residual(ctx, ora)
    d0, d1, _ = _steps_with_diagnostics(ctx, ora, 30, 0.0)
    assert abs(d1["mass"] - d0["mass"]) <= 1e-13 * d0["mass"]
    assert d1["r_cells"] == 1


def test_all_dry_domain():
    """every cell dry (the surface 20 m below the deepest point): zero
    residual, degree 0 everywhere, each cell moved to its dry-start level
    (Eq. initial_guess), no water or tracer created; the CFL step is bounded
    by the wave-speed floor, so the steps are huge but finite"""
    wl = W.closed_basin()
    wl.zeta = -20.0 * np.ones_like(wl.zeta)
    wl.qx[:] = 0.0
    wl.qy[:] = 0.0
    ctx, ora = pair(wl)
    rg = ctx.residual(0.0)
    for k, v in rg.items():
        assert not np.any(v), k
    tg = ctx.step(3, -1.0, 0.0)
    to = ora.step(3, -1.0, 0.0)
    assert np.isfinite(tg) and abs(tg - to) <= 1e-10 * to
    check_state(ctx, ora)
    dg = ctx.diagnostics()
    assert dg["mass"] == 0.0 and dg["tracer_mass"] == 0.0
    assert dg["r_cells"] == 0 and dg["positivity_violations"] == 0
    z = ctx.get_state()[0]
    assert np.all(z < 0.0)


def test_empty_mesh_is_rejected():
    """n = 0 cells: the context refuses the mesh with SWDG_EINVAL (nothing is
    launched); the allocation-free residual's refusal is checked on the CPU"""
    wl = W.closed_basin()
    ctx = swdg.Context(**wl.config())
    with pytest.raises(swdg.SwdgError) as e:
        ctx.upload_mesh(wl.mesh.x0y0[:0], wl.mesh.hxhy[:0], wl.mesh.nbr[:0])
    assert e.value.code == swdg.SWDG_EINVAL
