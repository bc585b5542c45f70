"""Pins of the step adjoint oracle (CPU).

``oracle/torch_step.py`` restates one fixed-size IMEX time step (degree
switch and remap, Newton continuity solve, momentum and tracer systems,
residuals, final combination) on top of the residual restatement.  Pinned
here against the independent C oracle: the states after the same fixed steps
agree to round-off, and the step's vector-Jacobian product (autograd along
the forward's path, each converged solve differentiated by the implicit
function theorem) matches central differences of the C oracle's steps in
random directions of the state, the Manning coefficients and per-cell
bathymetry offsets.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.oracle import Oracle  # noqa: E402
from oracle.torch_step import TorchStep, step_value, step_vjp  # noqa: E402
from paper_2505_18743_gb300 import workloads as W  # noqa: E402

import test_oracle_adjoint as A  # noqa: E402


def wetdry_beach():
    wl = W.tidal_beach(window=(236, 120, 6, 4), degree=2, pix=16)
    Xn, Yn = W.nodal_coordinates(wl.mesh, 2)
    rng = np.random.default_rng(5)
    wl.zeta = 0.2 + 0.05 * np.sin(Xn / 300.0) + 0.005 * rng.standard_normal(Xn.shape)
    wl.qx = 0.05 * np.cos(Yn / 200.0) + 0.01 * rng.standard_normal(Xn.shape)
    wl.qy = 0.01 * rng.standard_normal(Xn.shape)
    wl.c = 0.5 + 0.3 * np.sin(Xn / 300.0 + Yn / 500.0)
    wl.manning = rng.uniform(0.01, 0.04, wl.mesh.n)
    return wl


CASES = {
    "beach_r2": lambda: A.beach(2),
    "beach_r3": lambda: A.beach(3, window=(236, 120, 4, 3)),
    "beach_P": lambda: A.beach(2, mode=1),
    "wetdry": wetdry_beach,
    "forest_r1": lambda: A.forest(1),
    "diffusion": A.diffusive_beach,
}


def oracle_steps(wl, state, manning, delta, dt, nsteps):
    ras = A.shifted_raster(wl, delta) if np.any(delta) else wl.raster
    o = Oracle(wl.mesh, ras, **wl.config())
    for (tag, kind, amp, per, ph) in wl.boundaries:
        o.set_boundary(tag, kind, amp, per, ph)
    o.set_manning(manning)
    if wl.tracer_diffusivity is not None:
        o.set_tracer_diffusivity(wl.tracer_diffusivity)
    o.set_state(*state)
    o.step(nsteps, dt, 0.0)
    return o.get_state()


def fixed_dt(wl):
    return 0.5 * Oracle.from_workload(wl).cfl_dt(0.0)


@pytest.mark.parametrize("case", sorted(CASES))
def test_torch_step_matches_the_c_oracle(case):
    wl = CASES[case]()
    dt = fixed_dt(wl)
    n = wl.mesh.n
    got = step_value(TorchStep(wl), wl.state(), wl.manning, np.zeros(n), 0.0, dt, 2)
    ref = oracle_steps(wl, wl.state(), wl.manning, np.zeros(n), dt, 2)
    for a, b in zip(got, ref):
        assert np.abs(a - b).max() <= 1e-11 * max(np.abs(b).max(), 1e-2)


def step_directional_check(wl, ndir, use_delta, nsteps=1, seed=3, h=1e-5, tol=1e-6):
    dt = fixed_dt(wl)
    rng = np.random.default_rng(seed)
    n, nd = wl.mesh.n, (wl.degree + 1) ** 2
    state = [np.array(a, dtype=np.float64) for a in wl.state()]
    man = np.array(wl.manning, dtype=np.float64)
    zero = np.zeros(n)
    base = oracle_steps(wl, state, man, zero, dt, nsteps)
    cot = [rng.standard_normal((n, nd)) / max(float(np.abs(b).max()), 1e-3) for b in base]
    bars = step_vjp(TorchStep(wl), state, man, zero, cot, 0.0, dt, nsteps)
    for _ in range(ndir):
        v = [rng.standard_normal((n, nd)) * 1e-2 for _ in range(4)]
        vn = rng.uniform(0.0, 1.0, n) * 1e-2
        vd = rng.standard_normal(n) * 1e-2 if use_delta else zero
        sp = oracle_steps(wl, [a + h * b for a, b in zip(state, v)], man + h * vn, h * vd, dt, nsteps)
        sm = oracle_steps(wl, [a - h * b for a, b in zip(state, v)], man - h * vn, -h * vd, dt, nsteps)
        fd = sum(float((c * (p - m)).sum()) for c, p, m in zip(cot, sp, sm)) / (2 * h)
        ad = sum(float((b * a).sum()) for b, a in zip(bars[:4], v)) + \
            float((bars[4] * vn).sum()) + float((bars[5] * vd).sum())
        assert abs(fd - ad) <= tol * max(abs(ad), 1e-12), (fd, ad)


def test_step_vjp_matches_central_differences_mode_S():
    step_directional_check(A.beach(2), 4, True)


def test_step_vjp_matches_central_differences_two_steps_r3():
    step_directional_check(A.beach(3, window=(236, 120, 4, 3)), 3, True, nsteps=2, seed=9)


def test_step_vjp_matches_central_differences_with_a_wet_dry_cell():
    wl = wetdry_beach()
    o = Oracle.from_workload(wl)
    o.degree_switch()
    assert (o.flags() == 0).sum() >= 1  # at least one r_K = 0 cell takes the scalar path
    step_directional_check(wl, 4, True, seed=4)


def test_step_vjp_matches_central_differences_mode_P():
    step_directional_check(A.beach(2, mode=1), 3, False, seed=6)


def test_step_vjp_matches_central_differences_on_a_2to1_forest():
    step_directional_check(A.forest(1), 3, True, seed=8)
