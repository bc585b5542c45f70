"""Discrete adjoint of the residual on the GPU (swdg_residual_vjp) against
the adjoint oracle (autograd of the PyTorch restatement, itself pinned to
central differences of the C oracle): every cotangent -- state, Manning
coefficient, bathymetry offset -- within 1e-11 of its scale, on conforming,
boundary and 2:1 faces, modes S and P, degrees 1-3.

On a flat bottom the reconstruction's min(V_own(zeta), V_nb(zeta)) sits on
exact ties, where the bathymetry derivative is one-sided and which side a
tie takes is decided by the rounding of V (the library's deep-water shortcut
against the oracle's pixel sum): there the offset cotangent is not compared.
"""
import numpy as np
import pytest

from oracle.torch_residual import TorchResidual, residual_vjp
from paper_2505_18743_gb300 import swdg
from paper_2505_18743_gb300 import workloads as W

import test_oracle_adjoint as A

pytestmark = pytest.mark.gpu

VJP_TOL = 1e-11
KEYS = ("zeta", "qx", "qy", "c", "manning", "delta")


@pytest.fixture(scope="module", autouse=True)
def _build():
    import torch
    assert torch.cuda.is_available()
    from paper_2505_18743_gb300 import build as B
    from oracle import oracle
    B.build()
    oracle.build()


def compare(wl, t=1000.0, seed=2, precision=0, check_delta=True):
    n, nd = wl.mesh.n, (wl.degree + 1) ** 2
    rng = np.random.default_rng(seed)
    cot = [rng.standard_normal((n, nd)) for _ in range(6)]
    man = wl.manning if wl.manning is not None else np.zeros(n)
    tr = TorchResidual(wl.mesh, wl.raster, wl.degree, wl.subgrid_mode, wl.g, wl.eps_vel,
                       wl.boundaries, wl.tracer_diffusivity)
    ref = residual_vjp(tr, wl.state(), man, np.zeros(n), cot, t)
    ctx = swdg.Context.from_workload(wl, precision=precision)
    got = ctx.residual_vjp(cot, t)
    ctx.close()
    errs = {}
    for key, r in zip(KEYS, ref):
        if key == "delta" and not check_delta:
            continue
        scale = max(float(np.abs(r).max()), 1e-300)
        errs[key] = float(np.abs(got[key] - r).max()) / scale
        assert errs[key] <= VJP_TOL, (key, errs)
    return errs


@pytest.mark.parametrize("case", ["basin", "beach_r1", "beach_r2", "beach_r3", "beach_P",
                                  "forest_r1", "forest_r2", "diffusion"])
def test_residual_vjp_matches_the_adjoint_oracle(case):
    wl = {"basin": lambda: W.closed_basin(), "beach_r1": lambda: A.beach(1),
          "beach_r2": lambda: A.beach(2), "beach_r3": lambda: A.beach(3),
          "beach_P": lambda: A.beach(2, mode=1), "forest_r1": lambda: A.forest(1),
          "forest_r2": lambda: A.forest(2), "diffusion": A.diffusive_beach}[case]()
    compare(wl, check_delta=case != "basin")  # the basin's bottom is flat in places


def test_residual_vjp_is_fp64_in_an_fp32_bulk_context():
    compare(A.beach(2), precision=1)


def test_residual_vjp_with_dry_cells_and_friction():
    wl = W.lake_at_rest_bump(n=6, pix=4, degree=2, submerged=False)
    Xn, Yn = W.nodal_coordinates(wl.mesh, 2)
    wl.zeta = 0.05 * np.sin(3 * Xn) * np.cos(5 * Yn)
    wl.qx = 0.01 * np.cos(4 * Yn) + 0.0 * Xn
    wl.manning = np.full(wl.mesh.n, 0.03)
    compare(wl, t=0.0, check_delta=False)  # flat floor away from the bump


def test_residual_vjp_at_exact_wave_speed_ties():
    """the checkerboard case (exact wave-speed ties with discharge jumps at
    every interior face): the symmetric subgradient of the oracle, under two
    numberings of the cells"""
    wl = A.checkerboard_ties()
    compare(wl, t=0.0, check_delta=False)  # flat bottom: one-sided offset derivative
    perm = np.random.default_rng(13).permutation(wl.mesh.n)
    compare(A.renumbered_workload(wl, perm), t=0.0, check_delta=False)
