"""torch.autograd through K time steps of the CUDA path (adjoint.solve):
gradients with respect to the Manning coefficients, per-cell bathymetry
offsets and the start state against central differences of the CUDA forward
in 20 random directions, against the step adjoint oracle over three steps,
and independent of the checkpoint interval."""
import numpy as np
import pytest

from oracle.torch_step import TorchStep, step_vjp
from paper_2505_18743_gb300 import adjoint, swdg
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


def shore_case():
    # the shoreline band of the beach with an f64 raster (offsets exact), wet and dry cells
    wl = W.tidal_beach(window=(236, 120, 6, 4), degree=2, pix=16, dtype=np.float64)
    Xn, Yn = W.nodal_coordinates(wl.mesh, 2)
    rng = np.random.default_rng(4)
    wl.zeta = 0.3 + 0.05 * np.sin(Xn / 300.0) + 0.005 * rng.standard_normal(Xn.shape)
    wl.qx = 0.05 * np.cos(Yn / 200.0) + 0.01 * rng.standard_normal(Xn.shape)
    wl.qy = 0.01 * rng.standard_normal(Xn.shape)
    wl.c = 0.5 + 0.3 * np.sin(Xn / 300.0 + Yn / 500.0)
    wl.manning = rng.uniform(0.015, 0.035, wl.mesh.n)
    return wl


def tensors(wl, torch, grad=True):
    dev = torch.device("cuda")
    mk = lambda a: torch.tensor(np.asarray(a, dtype=np.float64), device=dev, requires_grad=grad)
    return [mk(a) for a in wl.state()], mk(wl.manning), mk(np.zeros(wl.mesh.n))


def objective(outs, w):
    return sum((o * wi).sum() for o, wi in zip(outs, w))


def test_gradients_match_central_differences_through_25_steps():
    torch = pytest.importorskip("torch")
    wl = shore_case()
    ctx = swdg.Context.from_workload(wl)
    dt = 0.5 * ctx.cfl_dt(0.0)
    state, man, delta = tensors(wl, torch)
    n, nd = wl.mesh.n, 9
    rng = np.random.default_rng(8)
    w = [torch.tensor(rng.standard_normal((n, nd)), device="cuda") for _ in range(4)]
    outs = adjoint.solve(ctx, *state, man, delta, nsteps=25, dt=dt, checkpoint_every=10)
    objective(outs, w).backward()
    grads = [s.grad for s in state] + [man.grad, delta.grad]
    assert all(g is not None and torch.isfinite(g).all() for g in grads)

    def J(v, h):
        with torch.no_grad():
            st = [s + h * d for s, d in zip(state, v[:4])]
            o = adjoint.solve(ctx, *st, man + h * v[4], delta + h * v[5], nsteps=25, dt=dt,
                              checkpoint_every=10)
            return float(objective(o, w))

    # central differences in 20 random directions of (state, n, delta); the error
    # is measured against the sum of the absolute per-parameter contributions,
    # the scale at which the central difference carries round-off
    worst = 0.0
    for _ in range(20):
        v = [torch.tensor(rng.standard_normal((n, nd)) * 1e-2, device="cuda") for _ in range(4)]
        v.append(torch.tensor(rng.uniform(0.0, 1.0, n) * 1e-3, device="cuda"))
        v.append(torch.tensor(rng.standard_normal(n) * 1e-2, device="cuda"))
        h = 1e-4
        fd = (J(v, h) - J(v, -h)) / (2 * h)
        parts = [float((g * d).sum()) for g, d in zip(grads, v)]
        err = abs(fd - sum(parts)) / sum(abs(p) for p in parts)
        worst = max(worst, err)
    assert worst <= 1e-5, worst


def test_gradients_match_the_step_adjoint_oracle_over_three_steps():
    torch = pytest.importorskip("torch")
    wl = shore_case()
    ctx = swdg.Context.from_workload(wl)
    dt = 0.5 * ctx.cfl_dt(0.0)
    state, man, delta = tensors(wl, torch)
    rng = np.random.default_rng(12)
    cot = [rng.standard_normal((wl.mesh.n, 9)) for _ in range(4)]
    outs = adjoint.solve(ctx, *state, man, delta, nsteps=3, dt=dt, checkpoint_every=2)
    objective(outs, [torch.tensor(c, device="cuda") for c in cot]).backward()
    got = [s.grad.cpu().numpy() for s in state] + [man.grad.cpu().numpy(), delta.grad.cpu().numpy()]
    ref = step_vjp(TorchStep(wl), wl.state(), wl.manning, np.zeros(wl.mesh.n), cot, 0.0, dt, 3)
    for a, b in zip(got, ref):
        assert np.abs(a - b).max() <= 1e-9 * max(np.abs(b).max(), 1e-300)


def test_checkpoint_interval_does_not_change_gradients():
    torch = pytest.importorskip("torch")
    wl = shore_case()
    grads = []
    for every in (1, 4, 30):
        ctx = swdg.Context.from_workload(wl)
        state, man, delta = tensors(wl, torch)
        outs = adjoint.solve(ctx, *state, man, delta, nsteps=9, dt=-1.0, checkpoint_every=every)
        (outs[0].sum() + outs[3].square().sum()).backward()
        grads.append([s.grad.clone() for s in state] + [man.grad.clone(), delta.grad.clone()])
        ctx.close()
    for g in grads[1:]:
        for a, b in zip(g, grads[0]):
            assert torch.equal(a, b)
