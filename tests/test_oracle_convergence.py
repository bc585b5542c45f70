"""Order-of-convergence pins of the oracle against closed-form solutions:
the travelling vortex of Sec. 4.4 (design order r+1, Table tab:vortex_metric)
and the Manning friction decay of a uniform stream (Eq. manning with the
IMEX TR-BDF2 part of Appendix A, second order in time)."""
import numpy as np
import pytest
from scipy.integrate import quad

from helpers import Vortex, cell_quadrature, golden_rows, vortex_H
from oracle.oracle import Oracle
from paper_2505_18743_gb300 import workloads as W


def test_vortex_primitive_is_the_cyclostrophic_integral():
    """H(x) printed in Sec. 4.4 is a primitive of x cos^8(x), which makes the
    vortex depth satisfy g dh/dR = R omega^2 (cyclostrophic balance)."""
    for a, b in [(0.0, 0.7), (0.3, np.pi / 2), (0.0, np.pi / 2)]:
        val, _ = quad(lambda x: x * np.cos(x) ** 8, a, b, epsabs=1e-14)
        assert abs((vortex_H(b) - vortex_H(a)) - val) < 1e-13


def vortex_error(N, degree, tableau, cfl):
    v = Vortex()
    mesh, ras = W.flat_periodic(2 * N, N, v.Lx, v.Ly, v.h0, degree, pix=1)
    X, Y = W.nodal_coordinates(mesh, degree)
    h, u, w = v(X, Y, 0.0)
    o = Oracle(mesh, ras, degree=degree, tableau=tableau, cfl=cfl, eps_vel=1e-3, h_lim=1e-3)
    o.set_state(h - v.h0, h * u, h * w, np.ones_like(h))
    nst = int(np.ceil(v.T / o.cfl_dt()))
    o.step(nst, v.T / nst)
    px, py, wt = cell_quadrature(mesh, 6)
    zeta = o.gauges(np.stack([px, py], 1))
    he, _, _ = v(px, py, v.T)
    return float(np.sqrt(np.sum(wt * (zeta - (he - v.h0)) ** 2)))


def paper_vortex(r, nmax):
    for row in golden_rows("vortex_static.txt"):
        if int(row[0]) == r and int(row[2]) == nmax:
            return float(row[4])
    raise KeyError


def test_vortex_degree2_ssp33_third_order_and_paper_value():
    e10 = vortex_error(10, 2, 1, 0.1)
    e20 = vortex_error(20, 2, 1, 0.1)
    assert np.log2(e10 / e20) > 2.7  # design order r + 1 = 3
    assert abs(e20 / paper_vortex(2, 1) - 1.0) < 0.25  # 1.125e-4 printed at N = 20


@pytest.mark.slow
def test_vortex_degree1_rk32_second_order_and_paper_value():
    e20 = vortex_error(20, 1, 0, 0.25)
    e40 = vortex_error(40, 1, 0, 0.25)
    assert np.log2(e20 / e40) > 1.8  # design order 2
    assert 0.5 < e20 / paper_vortex(1, 1) < 2.0  # 2.459e-3 printed at N = 20


def friction_run(dt, T, n_man, q0=1.5, h0=2.0, degree=1, tableau=0):
    # 1 km cells: the gravity-wave CFL stays below 0.05 for every step used here
    mesh, ras = W.flat_periodic(3, 3, 3000.0, 3000.0, h0, degree, pix=2)
    o = Oracle(mesh, ras, degree=degree, tableau=tableau, eps_vel=0.01)
    o.set_manning(np.full(mesh.n, n_man))
    nd = (degree + 1) ** 2
    one = np.ones((mesh.n, nd))
    o.set_state(0 * one, q0 * one, 0 * one, one)
    nst = int(round(T / dt))
    qs = []
    for _ in range(nst):
        o.step(1, dt)
        qs.append(o.get_state()[1][0, 0])
    return np.array(qs)


def test_manning_friction_converges_to_closed_form():
    """uniform stream: dq/dt = -g n^2 |q| q / h^(7/3), so q(t) = q0 / (1 + k q0 t)
    with k = g n^2 / h^(7/3).  Taken explicitly (SSP33) the friction term is
    third order in time; in the IMEX scheme the implicit diagonal uses the
    coefficient of the previous stage, gamma(q^(l-1)) (Eqs. imex_shw,
    mass_matrix_discharge), which makes it first order."""
    g, n_man, q0, h0, T = 9.81, 0.08, 1.5, 2.0, 40.0
    k = g * n_man ** 2 / h0 ** (7.0 / 3.0)
    exact = q0 / (1 + k * q0 * T)
    e = [abs(friction_run(T / m, T, n_man, tableau=1)[-1] - exact) for m in (8, 16, 32)]
    assert e[0] / e[1] > 7.0 and e[1] / e[2] > 7.5
    e = [abs(friction_run(T / m, T, n_man, tableau=0)[-1] - exact) for m in (8, 16, 32, 64)]
    for i in range(3):
        assert 1.9 < e[i] / e[i + 1] < 2.2
    assert e[-1] < 3e-4 * q0


def test_stiff_friction_is_stable_with_large_steps():
    """n = 1 (the paper's strong-friction channel): with dt twenty times the
    relaxation time the L-stable implicit part keeps q bounded and decaying
    to the right asymptote (an explicit treatment diverges here)."""
    g, q0, h0 = 9.81, 1.5, 2.0
    k = g * 1.0 / h0 ** (7.0 / 3.0)
    tau = 1.0 / (k * q0)  # initial relaxation time
    qs = friction_run(20 * tau, 400 * tau, 1.0)
    assert np.all(np.abs(qs) <= q0)
    assert np.all(np.abs(qs[5:]) <= np.abs(qs[4]))
    exact = q0 / (1 + k * q0 * 400 * tau)
    assert abs(qs[-1] - exact) < 0.15 * exact
