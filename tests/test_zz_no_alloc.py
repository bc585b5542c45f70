"""The allocation-free residual (swdg_residual_noalloc) against the FP64
oracle and against the context residual (swdg_residual + swdg_cfl_dt),
through the C-ABI, on two calls in a row.  It is for callers that cannot
allocate device memory (a memory pool that forbids new allocations, a device
whose memory is already reserved), so it takes every buffer from the caller
and keeps its scratch in a fixed array of the library; the free device
memory is checked to stay unchanged across a call.
"""
import numpy as np
import pytest

from helpers import residual_errors
from oracle.oracle import Oracle
from paper_2505_18743_gb300 import swdg
from paper_2505_18743_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12  # the residual tolerance of the parity tests


def tiles_of(wl):
    """the [n][P][P] per-cell pixel tiles of a cell-aligned raster (input
    preparation: a reshape of the raster, no method arithmetic)"""
    r = wl.raster
    P = int(round(wl.mesh.hxhy[0, 0] / r.dx))
    i0 = np.rint((wl.mesh.x0y0[:, 0] - r.xo) / r.dx).astype(int)
    j0 = np.rint((wl.mesh.x0y0[:, 1] - r.yo) / r.dy).astype(int)
    t = np.stack([r.z[j:j + P, i:i + P] for i, j in zip(i0, j0)])
    return np.ascontiguousarray(t), P


def run_case(wl, states, t):
    import torch
    dev = torch.device("cuda", 0)
    ctx = swdg.Context.from_workload(wl)
    tiles, P = tiles_of(wl)
    pix = swdg.SWDG_PIX_F32 if tiles.dtype == np.float32 else swdg.SWDG_PIX_F64
    n, nd = wl.mesh.n, (wl.degree + 1) ** 2
    d_hxhy = torch.tensor(wl.mesh.hxhy, dtype=torch.float64, device=dev).contiguous()
    d_nbr = torch.tensor(wl.mesh.nbr, dtype=torch.int32, device=dev).contiguous()
    d_tiles = torch.from_numpy(tiles).to(dev).contiguous()
    man = wl.manning if wl.manning is not None else np.zeros(n)
    d_man = torch.tensor(man, dtype=torch.float64, device=dev)
    d_res = torch.empty((6, n, nd), dtype=torch.float64, device=dev)
    d_dt = torch.empty(1, dtype=torch.float64, device=dev)
    cfg = swdg.swdg_config(wl.degree, 0, 0, wl.tableau, wl.g, wl.eps_vel, wl.h_lim, wl.eps0,
                           wl.cfl, 20, 1e-12, torch.cuda.current_stream(dev).cuda_stream)
    ora = Oracle.from_workload(wl)
    d_states = [torch.tensor(np.stack(st), dtype=torch.float64, device=dev).contiguous()
                for st in states]
    torch.cuda.synchronize(dev)
    for call, (st, d_state) in enumerate(zip(states, d_states)):
        # two calls in a row share the library's scratch
        ctx.set_state(*st)
        ref = ctx.residual(t)
        dt_ref = ctx.cfl_dt(t)
        ora.set_state(*st)
        ro = ora.residual(t)
        dt_ora = ora.cfl_dt(t)
        torch.cuda.synchronize(dev)
        free0, _ = torch.cuda.mem_get_info(dev)
        swdg.residual_noalloc(cfg, n, d_hxhy, d_nbr, d_tiles, P, pix, d_man, d_state, t, d_res,
                              d_dt, bc=wl.boundaries)
        torch.cuda.synchronize(dev)
        free1, _ = torch.cuda.mem_get_info(dev)
        if call > 0:  # the first call may still load the library's device code
            assert free1 == free0, (free0, free1)
        got = dict(zip(("F", "Gx", "Gy", "R", "Lx", "Ly"), d_res.cpu().numpy()))
        err_ora = residual_errors(got, ro)
        assert max(err_ora.values()) <= TOL, err_ora
        err_ctx = residual_errors(got, ref)
        assert max(err_ctx.values()) <= TOL, err_ctx
        dt = float(d_dt.item())
        assert abs(dt - dt_ora) <= 1e-13 * dt_ora and abs(dt - dt_ref) <= 1e-13 * dt_ref
    ctx.close()


def perturbed(st, seed):
    rng = np.random.default_rng(seed)
    return tuple(a + 0.01 * rng.standard_normal(a.shape) for a in st)


def test_noalloc_residual_matches_context_closed_basin():
    wl = W.closed_basin()
    s0 = wl.state()
    run_case(wl, [s0, perturbed(s0, 1)], 0.0)


def test_noalloc_residual_matches_context_tidal_beach_crop():
    wl = W.tidal_beach(window=(0, 120, 12, 10))
    Xn, Yn = W.nodal_coordinates(wl.mesh, 3)
    # every field varies in x and y, so each residual field carries signal
    s0 = (0.3 * np.sin(Xn / 400.0) * np.cos(Yn / 300.0), 0.2 * np.cos(Yn / 200.0),
          0.1 * np.sin(Xn / 250.0), wl.c)
    run_case(wl, [s0, perturbed(s0, 2)], 1500.0)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    dev = torch.device("cuda", 0)
    one = torch.zeros(16, dtype=torch.float64, device=dev)
    cfg = swdg.swdg_config(1, 0, 0, 0, 9.81, 0.01, 0.01, 1e-6, 0.1, 20, 1e-12, None)
    with pytest.raises(swdg.SwdgError) as e:
        swdg.residual_noalloc(cfg, 1048577, one, one, one, 8, swdg.SWDG_PIX_F64, one, one, 0.0,
                              one, one)
    assert e.value.code == swdg.SWDG_EINVAL
    assert "1048576" in str(e.value)
    # only the FP64 residual exists without a context: FP32-bulk is refused
    cfg32 = swdg.swdg_config(1, 1, 0, 0, 9.81, 0.01, 0.01, 1e-6, 0.1, 20, 1e-12, None)
    with pytest.raises(swdg.SwdgError) as e:
        swdg.residual_noalloc(cfg32, 1, one, one, one, 8, swdg.SWDG_PIX_F64, one, one, 0.0,
                              one, one)
    assert e.value.code == swdg.SWDG_EINVAL and "precision" in str(e.value)
