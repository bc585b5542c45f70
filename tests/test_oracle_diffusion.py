"""Pins of the tracer numerical diffusion in the oracle (Eq. numdiff: the
term -sum_K int_K nu_c h grad c . grad psi_i added to the tracer residual R).

The term vanishes for a constant tracer, sums to zero over each cell (it
moves no tracer mass), is dissipative (<c, R_diff> = -int nu_c h |grad c|^2
<= 0 on every cell), and for a linear tracer a x + b y over a flat wet
bottom of depth h its first moments are sum_i x_i R_diff,i = -nu_c h a |K|
and sum_i y_i R_diff,i = -nu_c h b |K| (the nodal coordinates reproduce x and
y, so sum_i x_i grad psi_i = grad x)."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2505_18743_gb300 import workloads as W


def resid_diff(wl, nu):
    o0 = Oracle.from_workload(wl)
    o1 = Oracle.from_workload(wl)
    o1.set_tracer_diffusivity(nu)
    return o1.residual(0.0)["R"] - o0.residual(0.0)["R"], o0.residual(0.0)["R"]


def beach(degree):
    wl = W.tidal_beach(window=(232, 120, 6, 5), degree=degree, pix=16)
    Xn, Yn = W.nodal_coordinates(wl.mesh, degree)
    wl.zeta = 0.2 + 0.1 * np.sin(Xn / 300.0)
    wl.qx = 0.1 * np.cos(Yn / 200.0) + 0.0 * Xn
    wl.c = 0.5 + 0.4 * np.sin(Xn / 150.0) * np.cos(Yn / 120.0)
    return wl


@pytest.mark.parametrize("degree", [1, 2, 3])
def test_diffusion_is_conservative_and_dissipative(degree):
    wl = beach(degree)
    nu = np.linspace(1.0, 5.0, wl.mesh.n)
    rd, r0 = resid_diff(wl, nu)
    scale = np.abs(rd).max()
    assert scale > 1e-6 * np.abs(r0).max()            # the term is present
    assert np.abs(rd.sum(1)).max() <= 1e-12 * scale * rd.shape[1]
    assert np.all((wl.c * rd).sum(1) <= 1e-12 * scale)  # <c, R_diff> <= 0 per cell
    wl.c = np.full_like(wl.c, 0.7)
    rd, _ = resid_diff(wl, nu)
    assert np.abs(rd).max() <= 1e-12 * scale


@pytest.mark.parametrize("degree", [1, 2, 3])
def test_diffusion_moments_of_a_linear_tracer(degree):
    mesh, ras = W.flat_periodic(4, 3, 400.0, 300.0, 7.0, degree, pix=4)
    Xn, Yn = W.nodal_coordinates(mesh, degree)
    a, b = 0.003, -0.002
    zero = np.zeros_like(Xn)
    wl = W.Workload("flat", degree, mesh, ras, zero, zero.copy(), zero.copy(), a * Xn + b * Yn)
    nu = np.full(mesh.n, 2.5)
    rd, _ = resid_diff(wl, nu)
    J = mesh.hxhy[:, 0] * mesh.hxhy[:, 1]
    np.testing.assert_allclose((Xn * rd).sum(1), -2.5 * 7.0 * a * J, rtol=1e-12)
    np.testing.assert_allclose((Yn * rd).sum(1), -2.5 * 7.0 * b * J, rtol=1e-12)


def test_tracer_mass_is_kept_with_diffusion_over_steps():
    wl = W.closed_basin()
    wl.tracer_diffusivity = np.full(wl.mesh.n, 0.5)
    o = Oracle.from_workload(wl)
    d0 = o.diagnostics()
    o.step(30)
    d1 = o.diagnostics()
    assert abs(d1["tracer_mass"] - d0["tracer_mass"]) <= 1e-13 * d0["tracer_mass"]
    assert abs(d1["mass"] - d0["mass"]) <= 1e-13 * d0["mass"]
