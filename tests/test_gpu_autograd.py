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


def gauge_points(wl, ng, seed=2):
    rng = np.random.default_rng(seed)
    lo = wl.mesh.x0y0.min(0)
    hi = (wl.mesh.x0y0 + wl.mesh.hxhy).max(0)
    return np.stack([rng.uniform(lo[0], hi[0], ng), rng.uniform(lo[1], hi[1], ng)], 1)


def test_gauge_misfit_gradient_matches_central_differences():
    # loss = sum over 12 steps and 12 gauges of the squared zeta misfit against
    # a run with another Manning field; 20 random directions
    torch = pytest.importorskip("torch")
    wl = shore_case()
    ctx = swdg.Context.from_workload(wl)
    dt = 0.5 * ctx.cfl_dt(0.0)
    xy = gauge_points(wl, 12)
    state, man, delta = tensors(wl, torch)
    nsteps = 12
    with torch.no_grad():
        man_true = man * (1.0 + 0.3 * torch.sin(torch.arange(wl.mesh.n, device="cuda") * 0.7))
        *_, G_true = adjoint.solve(ctx, *state, man_true, delta, nsteps=nsteps, dt=dt, gauges=xy)
    *_, G = adjoint.solve(ctx, *state, man, delta, nsteps=nsteps, dt=dt, gauges=xy,
                          checkpoint_every=5)
    assert G.shape == (nsteps, 12) and bool(torch.isfinite(G).all())
    ((G - G_true) ** 2).sum().backward()
    grads = [s.grad for s in state] + [man.grad, delta.grad]
    assert float(man.grad.abs().max()) > 0

    def J(v, h):
        with torch.no_grad():
            st = [s + h * d for s, d in zip(state, v[:4])]
            *_, g = adjoint.solve(ctx, *st, man + h * v[4], delta + h * v[5], nsteps=nsteps, dt=dt,
                                  gauges=xy)
            return float(((g - G_true) ** 2).sum())

    rng = np.random.default_rng(3)
    n, nd = wl.mesh.n, 9
    worst = 0.0
    for _ in range(20):
        v = [torch.tensor(rng.standard_normal((n, nd)) * 1e-2, device="cuda") for _ in range(4)]
        v.append(torch.tensor(rng.uniform(0.0, 1.0, n) * 1e-3, device="cuda"))
        v.append(torch.tensor(rng.standard_normal(n) * 1e-2, device="cuda"))
        h = 1e-4
        fd = (J(v, h) - J(v, -h)) / (2 * h)
        parts = [float((g * d).sum()) for g, d in zip(grads, v)]
        worst = max(worst, abs(fd - sum(parts)) / sum(abs(p) for p in parts))
    assert worst <= 1e-5, worst


def test_gauge_misfit_gradient_matches_the_oracle():
    # the gauge values are a fixed linear map of the nodal zeta (the Lagrange
    # basis of each gauge's cell at its point): the oracle's loss over three
    # steps, differentiated by autograd of the step oracle
    torch = pytest.importorskip("torch")
    from oracle.amr import _lagrange
    from oracle.oracle import rule
    wl = shore_case()
    ctx = swdg.Context.from_workload(wl)
    dt = 0.5 * ctx.cfl_dt(0.0)
    ng = 9
    xy = gauge_points(wl, ng, seed=5)
    state, man, delta = tensors(wl, torch)
    rng = np.random.default_rng(6)
    target = torch.tensor(rng.standard_normal((3, ng)) * 0.05, device="cuda")
    *_, G = adjoint.solve(ctx, *state, man, delta, nsteps=3, dt=dt, gauges=xy, checkpoint_every=2)
    ((G - target) ** 2).sum().backward()
    got = [s.grad.cpu().numpy() for s in state] + [man.grad.cpu().numpy(), delta.grad.cpu().numpy()]
    xs, _ = rule(1, 3)
    Wg = np.zeros((ng, wl.mesh.n, 9))
    for g, (x, y) in enumerate(xy):
        lo, hx = wl.mesh.x0y0, wl.mesh.hxhy
        k = np.nonzero((lo[:, 0] <= x) & (x <= lo[:, 0] + hx[:, 0]) &
                       (lo[:, 1] <= y) & (y <= lo[:, 1] + hx[:, 1]))[0][0]
        xi, et = (x - lo[k, 0]) / hx[k, 0], (y - lo[k, 1]) / hx[k, 1]
        Wg[g, k] = np.outer(_lagrange(xs, et), _lagrange(xs, xi)).ravel()
    Wt = torch.tensor(Wg)
    ts = TorchStep(wl)
    u = [torch.tensor(np.asarray(a, dtype=np.float64), requires_grad=True) for a in wl.state()]
    m = torch.tensor(wl.manning, requires_grad=True)
    dl = torch.zeros(wl.mesh.n, dtype=torch.float64, requires_grad=True)
    cur, loss, tt = u, 0.0, 0.0
    for i in range(3):
        cur = ts.step(cur, m, dl, tt, dt)
        tt += dt
        Gi = torch.einsum("gkj,kj->g", Wt, cur[0])
        assert np.abs(Gi.detach().numpy() - G[i].detach().cpu().numpy()).max() <= 1e-9
        loss = loss + ((Gi - target[i].cpu()) ** 2).sum()
    ref = torch.autograd.grad(loss, u + [m, dl], allow_unused=True)  # c does not reach zeta
    for a, b, x in zip(got, ref, u + [m, dl]):
        b = np.zeros(x.shape) if b is None else b.numpy()
        if not np.abs(b).max() > 0:
            assert np.abs(a).max() == 0.0
            continue
        assert np.abs(a - b).max() <= 1e-9 * max(np.abs(b).max(), 1e-300)


def test_gauge_misfit_gradient_at_full_size():
    # the adjoint case at its full size (128 x 128 cells, r = 2, 16 x 16 px,
    # 50 gauges, 200 steps, checkpoint every 20), the CFL steps of a first run
    # held fixed.  Central differences along a bathymetry offset cross kinks
    # of the scheme (the hydrostatic reconstruction's max(z_L, z_R) over the
    # noisy bottom, the wet-pixel indicator) and so converge only as O(h):
    # 20 random directions in (state, Manning, offset) agree to 1e-3 of the
    # summed per-parameter contributions, directions in (state, Manning)
    # alone, which leave the bottom in place, to 1e-4.
    torch = pytest.importorskip("torch")
    wl, xy, man_true = W.gauge_misfit_case()
    ctx = swdg.Context.from_workload(wl)
    nsteps = 200
    ctx.set_manning(wl.manning)
    t, dts = 0.0, []
    for _ in range(nsteps):
        t = ctx.step(1, -1.0, t)
        dts.append(ctx.clock()[1])
    state, man, delta = tensors(wl, torch)
    with torch.no_grad():
        mt = torch.tensor(man_true, device="cuda")
        *_, G_true = adjoint.solve(ctx, *state, mt, delta, nsteps=nsteps, dt=dts, gauges=xy)
    *_, G = adjoint.solve(ctx, *state, man, delta, nsteps=nsteps, dt=dts, gauges=xy,
                          checkpoint_every=20)
    ((G - G_true) ** 2).sum().backward()
    grads = [s.grad for s in state] + [man.grad, delta.grad]
    assert all(bool(torch.isfinite(g).all()) for g in grads)
    assert float(man.grad.abs().max()) > 0 and float(delta.grad.abs().max()) > 0

    def J(v, h):
        with torch.no_grad():
            st = [s + h * d for s, d in zip(state, v[:4])]
            *_, g = adjoint.solve(ctx, *st, man + h * v[4], delta + h * v[5], nsteps=nsteps,
                                  dt=dts, gauges=xy)
            return float(((g - G_true) ** 2).sum())

    def err(v, h):
        fd = (J(v, h) - J(v, -h)) / (2 * h)
        parts = [float((g * d).sum()) for g, d in zip(grads, v)]
        return abs(fd - sum(parts)) / sum(abs(p) for p in parts)

    rng = np.random.default_rng(11)
    n, nd = wl.mesh.n, 9
    T = lambda a: torch.tensor(a, device="cuda")
    worst = 0.0
    for _ in range(20):
        v = [T(rng.standard_normal((n, nd)) * 1e-3) for _ in range(4)]
        v.append(T(rng.uniform(-1.0, 1.0, n) * 6e-3))
        v.append(T(rng.standard_normal(n) * 1e-2))
        worst = max(worst, err(v, 1e-3))
    assert worst <= 1e-3, worst
    for _ in range(3):
        v = [T(rng.standard_normal((n, nd)) * 1e-3) for _ in range(4)]
        v.append(T(rng.uniform(-1.0, 1.0, n) * 6e-3))
        v.append(torch.zeros(n, dtype=torch.float64, device="cuda"))
        assert err(v, 1e-3) <= 1e-4
