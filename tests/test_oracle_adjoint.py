"""Pins of the adjoint oracle (CPU).

``oracle/torch_residual.py`` restates the residual of Sec. 3.2 as PyTorch
tensor expressions so that autograd gives its exact vector-Jacobian product
(VJP).  It is pinned here against the independent C oracle twice: value for
value (the residuals agree to round-off on conforming, boundary and 2:1
faces, modes S and P), and derivative for derivative (for random
directions v in the state, the Manning coefficients and a per-cell
bathymetry offset, <R_bar, central difference of the C oracle along v> =
<VJP(R_bar), v>).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.oracle import Oracle  # noqa: E402
from oracle.torch_residual import TorchResidual, residual_value, residual_vjp  # noqa: E402
from paper_2505_18743_gb300 import workloads as W  # noqa: E402

FIELDS = ("F", "Gx", "Gy", "R", "Lx", "Ly")


def beach(degree=2, mode=0, window=(236, 120, 5, 4)):
    wl = W.tidal_beach(window=window, degree=degree, pix=16)
    wl.subgrid_mode = mode
    Xn, Yn = W.nodal_coordinates(wl.mesh, degree)
    rng = np.random.default_rng(7)
    wl.zeta = 0.3 * np.sin(Xn / 400.0) * np.cos(Yn / 300.0) + 0.01 * rng.standard_normal(Xn.shape)
    wl.qx = 0.2 * np.cos(Yn / 200.0) + 0.02 * rng.standard_normal(Xn.shape)
    wl.qy = 0.1 * np.sin(Xn / 250.0) + 0.02 * rng.standard_normal(Xn.shape)
    wl.c = 0.5 + 0.3 * np.sin(Xn / 300.0 + Yn / 500.0)
    wl.manning = rng.uniform(0.01, 0.04, wl.mesh.n)
    return wl


def forest(degree=1):
    wl = W.lagoon(nx0=8, ny0=4, pix0=8, degree=degree, levels=2, Lx=1600.0, Ly=800.0,
                  band=(400.0, 200.0))
    Xn, Yn = W.nodal_coordinates(wl.mesh, degree)
    rng = np.random.default_rng(3)
    # roughen the (flat at this scale) bottom: exact ties of the reconstruction's
    # min would make the bathymetry derivative one-sided
    z = np.asarray(wl.raster.z, dtype=np.float64)
    wl.raster = W.Raster(z + 0.05 * rng.standard_normal(z.shape), wl.raster.xo, wl.raster.yo,
                         wl.raster.dx, wl.raster.dy)
    wl.zeta = 0.2 * np.cos(Xn / 300.0) + 0.01 * rng.standard_normal(Xn.shape)
    wl.qx = 0.05 + 0.01 * rng.standard_normal(Xn.shape)
    wl.qy = 0.01 * rng.standard_normal(Xn.shape)
    wl.c = np.ones_like(Xn) + 0.1 * np.sin(Yn / 200.0)
    wl.manning = np.full(wl.mesh.n, 0.02)
    return wl


def torch_res(wl):
    return TorchResidual(wl.mesh, wl.raster, wl.degree, wl.subgrid_mode, wl.g, wl.eps_vel,
                         wl.boundaries, wl.tracer_diffusivity)


def diffusive_beach():
    wl = beach(2)
    wl.tracer_diffusivity = np.linspace(0.5, 3.0, wl.mesh.n)
    return wl


def shifted_raster(wl, delta):
    """the raster with every pixel of cell K deepened by delta_K (mode S)"""
    ras = wl.raster
    z = np.array(ras.z, dtype=np.float64)
    for k in range(wl.mesh.n):
        i0 = int(round((wl.mesh.x0y0[k, 0] - ras.xo) / ras.dx))
        j0 = int(round((wl.mesh.x0y0[k, 1] - ras.yo) / ras.dy))
        P = int(round(wl.mesh.hxhy[k, 0] / ras.dx))
        z[j0:j0 + P, i0:i0 + P] += delta[k]
    return W.Raster(z, ras.xo, ras.yo, ras.dx, ras.dy)


def c_residual(wl, state, manning, delta, t):
    ras = shifted_raster(wl, delta) if np.any(delta) else wl.raster
    o = Oracle(wl.mesh, ras, **wl.config())
    for (tag, kind, amp, per, ph) in wl.boundaries:
        o.set_boundary(tag, kind, amp, per, ph)
    o.set_manning(manning)
    if wl.tracer_diffusivity is not None:
        o.set_tracer_diffusivity(wl.tracer_diffusivity)
    o.set_state(*state)
    return o.residual(t)


@pytest.mark.parametrize("case", ["basin", "beach_r2", "beach_r3", "beach_P", "forest_r1", "forest_r2",
                                  "diffusion"])
def test_torch_residual_matches_the_c_oracle(case):
    wl = {"basin": lambda: W.closed_basin(), "beach_r2": lambda: beach(2),
          "diffusion": diffusive_beach,
          "beach_r3": lambda: beach(3), "beach_P": lambda: beach(2, mode=1),
          "forest_r1": lambda: forest(1), "forest_r2": lambda: forest(2)}[case]()
    t = 1000.0
    man = wl.manning if wl.manning is not None else np.zeros(wl.mesh.n)
    rv = residual_value(torch_res(wl), wl.state(), man, np.zeros(wl.mesh.n), t)
    ro = c_residual(wl, wl.state(), man, np.zeros(wl.mesh.n), t)
    scale = max(float(np.abs(v).max()) for v in ro.values())
    for k in FIELDS:
        assert np.abs(rv[k] - ro[k]).max() <= 1e-13 * scale, k


def directional_check(wl, ndir, use_delta, seed=11, t=1000.0, h=1e-4, tol=1e-6):
    tr = torch_res(wl)
    rng = np.random.default_rng(seed)
    n, nd = wl.mesh.n, (wl.degree + 1) ** 2
    state = [np.array(a, dtype=np.float64) for a in wl.state()]
    man = np.array(wl.manning, dtype=np.float64)
    delta = np.zeros(n)
    ro = c_residual(wl, state, man, delta, t)
    cot = [rng.standard_normal((n, nd)) / max(float(np.abs(ro[k]).max()), 1e-30) for k in FIELDS]
    bars = residual_vjp(tr, state, man, delta, cot, t)
    worst = 0.0
    for _ in range(ndir):
        v = [rng.standard_normal((n, nd)) * s for s in (1e-2, 1e-2, 1e-2, 1e-2)]
        vn = rng.uniform(0.0, 1.0, n) * 1e-2
        vd = rng.standard_normal(n) * 1e-2 if use_delta else np.zeros(n)
        rp = c_residual(wl, [a + h * b for a, b in zip(state, v)], man + h * vn, h * vd, t)
        rm = c_residual(wl, [a - h * b for a, b in zip(state, v)], man - h * vn, -h * vd, t)
        fd = sum(float((c * (rp[k] - rm[k])).sum()) for c, k in zip(cot, FIELDS)) / (2 * h)
        ad = sum(float((b * a).sum()) for b, a in zip(bars[:4], v)) + \
            float((bars[4] * vn).sum()) + float((bars[5] * vd).sum())
        err = abs(fd - ad) / max(abs(ad), 1e-12)
        worst = max(worst, err)
        assert err <= tol, (fd, ad, err)
    return worst


def test_vjp_matches_central_differences_mode_S_with_bathymetry_offset():
    directional_check(beach(2), 10, True)


def test_vjp_matches_central_differences_r3():
    directional_check(beach(3, window=(236, 120, 4, 3)), 5, True, seed=5)


def test_vjp_matches_central_differences_with_tracer_diffusion():
    directional_check(diffusive_beach(), 5, True, seed=19)


def test_vjp_matches_central_differences_mode_P():
    directional_check(beach(2, mode=1), 5, False, seed=13)


def test_vjp_matches_central_differences_on_a_2to1_forest():
    # many pixels sit near the waterline here: a smaller step keeps the
    # central differences from straddling the kinks of max(., 0)
    directional_check(forest(1), 5, True, seed=17, h=1e-5)


def test_vjp_is_finite_with_dry_cells_and_a_lake_at_rest():
    wl = W.lake_at_rest_bump(n=6, pix=4, degree=2, submerged=False)
    o = Oracle.from_workload(wl)
    z = o.lake_at_rest(0.0)
    zero = np.zeros_like(z)
    tr = torch_res(wl)
    n, nd = wl.mesh.n, z.shape[1]
    cot = [np.ones((n, nd))] * 6
    bars = residual_vjp(tr, [z, zero, zero, np.ones_like(z)], np.full(n, 0.03), np.zeros(n), cot)
    for b in bars:
        assert np.all(np.isfinite(b))
    # a fully dry cell (every pixel above the surface): no momentum sensitivity
    rv = residual_value(tr, [z, zero, zero, np.ones_like(z)], np.full(n, 0.03), np.zeros(n))
    assert np.abs(rv["F"]).max() < 1e-12


def renumbered(mesh, perm):
    """the mesh with old cell perm[i] as new cell i"""
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    nbr = mesh.nbr[perm].copy()
    nbr = np.where(nbr >= 0, inv[np.maximum(nbr, 0)], nbr).astype(np.int32)
    return W.Mesh(mesh.x0y0[perm].copy(), mesh.hxhy[perm].copy(), nbr)


def checkerboard_ties():
    """On a flat bottom, a continuous elevation with discharges whose sign
    flips from cell to cell (a checkerboard: the flows meet or part at every
    face) gives both sides of every interior face point the same wave-speed
    bound |u.n| + sqrt(g h) while the discharge jumps, so the maximum ties
    exactly where its derivative matters."""
    mesh, ras = W.flat_periodic(6, 5, 600.0, 500.0, 4.0, 1, pix=2, periodic=(False, False))
    X, Y = W.nodal_coordinates(mesh, 1)
    ij = np.rint((mesh.x0y0[:, 0] / 100.0) + (mesh.x0y0[:, 1] / 100.0)).astype(int)
    sgn = np.where(ij % 2 == 0, 1.0, -1.0)[:, None]
    zeta = 0.2 * np.sin(X / 170.0) * np.cos(Y / 130.0)
    qx = sgn * (0.3 + 0.2 * np.cos(Y / 90.0))
    qy = sgn * 0.1 * np.sin(X / 110.0)
    c = 0.5 + 0.3 * np.sin((X + Y) / 200.0)
    man = np.random.default_rng(11).uniform(0.01, 0.04, mesh.n)
    return W.Workload("checkerboard-ties", 1, mesh, ras, zeta, qx, qy, c, manning=man)


def renumbered_workload(wl, perm):
    m2 = renumbered(wl.mesh, perm)
    return W.Workload(wl.name + "-renumbered", wl.degree, m2, wl.raster,
                      *[a[perm] for a in wl.state()], manning=wl.manning[perm])


def test_vjp_at_wave_speed_ties_does_not_depend_on_cell_numbering():
    """At the exact ties of the checkerboard case the wave-speed maximum's
    derivative is the symmetric subgradient, which a renumbering of the
    cells (the same discrete operator) leaves unchanged; a rule that let the
    lower cell index decide would move derivative from one cell of the face
    to the other."""
    wl = checkerboard_ties()
    rng = np.random.default_rng(12)
    n, nd = wl.mesh.n, wl.zeta.shape[1]
    cot = [rng.standard_normal((n, nd)) for _ in range(6)]
    base = residual_vjp(torch_res(wl), wl.state(), wl.manning, np.zeros(n), cot)
    perm = rng.permutation(n)
    w2 = renumbered_workload(wl, perm)
    got = residual_vjp(torch_res(w2), w2.state(), w2.manning, np.zeros(n), [a[perm] for a in cot])
    for b, g in zip(base, got):
        scale = max(float(np.abs(b).max()), 1e-30)
        assert np.abs(g - b[perm]).max() <= 1e-13 * scale
