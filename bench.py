"""Benchmark of the sub-grid DG shallow-water hot path on GB300.

Workload: the 20 km tidal beach, degree-3 DG on a uniform 256 x 256 mesh,
16 x 16 pixels of a 4096 x 4096 float32 bathymetry per cell, RK32/TR-BDF2
IMEX with Manning friction, FP64 arithmetic.  One "step" = one time step of
the whole hot path: degree switch, three stages (residual + stage update) and
the final combination.

Metric: DoF-stage updates per second, where one DoF-stage update advances one
nodal value of (zeta, qx, qy, c) through one stage (residual + stage solve):
n_cells * 4 (r+1)^2 * 3 updates per step.  Inputs are larger than L2 (the
working set is about 0.5 GB), so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl swdg|reference]

N > 1 runs one independent replica per GPU and reports the whole-job rate
("weak" scaling): the path would shard by spatial domain with a face-trace
halo per stage, but each call here holds one GPU, so no exchange is built.
The reference arm (--impl reference) is the CPU oracle timed on the host's
cores on a bounded crop of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2505_18743_gb300 import workloads as W  # noqa: E402

METRIC = "DoF-stage updates/s"
WORKLOAD = "tidal-beach 256x256 cells, r=3, 16x16 px/cell (4096^2 f32 raster), RK32-IMEX, FP64"
STAGES = 3
# kernel-slot names of swdg_step_profile
SLOTS = ["step_begin", "residual_1", "residual_2", "residual_3", "residual_4", "stage_2",
         "stage_3", "stage_4", "final", "faces_1", "faces_2", "faces_3", "faces_4"]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def units_per_step(wl):
    nd = (wl.degree + 1) ** 2
    return wl.mesh.n * 4 * nd * STAGES


COUNTERS = os.path.join(ROOT, "profiles", "counters_tidal_beach_256x256_r3.txt")


def kernel_sources_hash():
    """sha256 (first 16 hex digits) over the CUDA sources, name and bytes of
    each file of the package's csrc/ in name order"""
    import hashlib
    d = os.path.join(ROOT, "paper_2505_18743_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(os.listdir(d)):
        h.update(f.encode())
        h.update(b"\0")
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def load_counters(path=COUNTERS):
    """the ncu counters of one step's launches (profiles/counters_...txt):
    ({precision: {slot: (fp64 flops per cell, fp32 flops per cell, DRAM bytes
    per launch)}}, whether they were taken on the current kernel sources).
    The kernels here are bound by the FP64 pipe, so the FP64 flops per cell
    give the roofline's achieved rate."""
    table, sha = {}, None
    with open(path) as f:
        for line in f:
            parts = line.split()
            if not parts or parts[0].startswith("#"):
                continue
            if parts[0] == "sources_sha256_16":
                sha = parts[1]
                continue
            prec, slot, f64, f32, dram = parts[:5]
            table.setdefault(prec, {})[slot] = (float(f64), float(f32), float(dram))
    return table, sha == kernel_sources_hash()


FP64_PEAK_TFLOPS = 1.25  # nominal GB300 FP64 (152 SMs x 2.07 GHz x 2 DFMA/clk x 2), if no probe


def measured_pipe_peaks():
    """the FP64 and FP32 FMA-chain peaks of this GPU, measured now by the
    library's probe (swdg_probe_fma): {dtype: (TFLOP/s, ms)}"""
    from paper_2505_18743_gb300 import swdg
    out = {}
    for name, code in (("fp64", swdg.SWDG_PIX_F64), ("fp32", swdg.SWDG_PIX_F32)):
        try:
            out[name] = swdg.probe_fma(code)
        except swdg.SwdgError:
            pass
    return out


def algorithmic_bytes_per_cell(kernel, r=3, P=16, pix_bytes=4, nres=3):
    """Algorithmic bytes one launch must move per cell (each input read once,
each output written once; intermediates that a fused path would keep on
chip -- the face slots -- are left out):
    residual: own state 4 nd f64 in, 6 nd f64 out, the pixel tile, geometry;
    stage update: v^n in, H/C~ in, nres residual sets of 6 nd in, state out."""
    nd = (r + 1) ** 2
    geo = 16 + 32 + 8 + 1
    if kernel.startswith("residual"):
        return 4 * nd * 8 + 6 * nd * 8 + P * P * pix_bytes + geo
    if kernel.startswith("faces"):  # the state once; the face slots are an intermediate
        return 4 * nd * 8 + geo
    if kernel.startswith("stage") or kernel == "final":
        return 4 * nd * 8 + 2 * nd * 8 + 16 + nres * 6 * nd * 8 + 4 * nd * 8 + geo
    return 4 * nd * 8 + 2 * nd * 8 + 16 + P * P * pix_bytes + geo


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region"""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def dist_init(n_gpus):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def omp_threads(k):
    """set the OpenMP thread count of the oracle's runtime (libgomp); False if
    the runtime cannot be reached"""
    import ctypes
    try:
        ctypes.CDLL("libgomp.so.1").omp_set_num_threads(int(k))
        return True
    except (OSError, AttributeError):
        return False


def cpu_oracle_rate(seconds=15.0, window=(184, 120, 24, 24)):
    """the oracle (as it stands) on a crop of the workload, steps until about
    `seconds` of CPU work; returns (updates/s, cores, sample text)"""
    from oracle.oracle import Oracle
    wl = W.tidal_beach(window=window)
    o = Oracle.from_workload(wl)
    t = 0.0
    n = 0
    t0 = time.perf_counter()
    while True:
        t = o.step(1, -1.0, t)
        n += 1
        if time.perf_counter() - t0 > seconds or n >= 5000:
            break
    el = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    rate = units_per_step(wl) * n / el
    sample = (f"{n} RK32 steps of the {window[2]}x{window[3]}-cell crop at cell ({window[0]},"
              f"{window[1]}) of the same workload ({wl.mesh.n} cells, the shoreline band), "
              f"{el:.1f} s")
    return rate, cores, sample


def run_reference(args, rank, world):
    if rank != 0:
        return
    os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
    per = []
    from oracle.oracle import Oracle
    wl = W.tidal_beach(window=(184, 120, 16, 16))
    o = Oracle.from_workload(wl)
    t = 0.0
    for _ in range(args.warmup):
        t = o.step(1, -1.0, t)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s0 = time.perf_counter()
        t = o.step(1, -1.0, t)
        per.append(time.perf_counter() - s0)
    el = time.perf_counter() - t0
    rate = units_per_step(wl) * args.steps / el
    cores = int(os.environ["OMP_NUM_THREADS"])
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": "updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "16x16-cell crop (184,120), CPU oracle"},
            "cpu_baseline": {"value": rate, "unit": "updates/s", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} RK32 steps of a 16x16-cell crop of the "
                                       "workload (cells 184..199 x 120..135)"},
            "e2e": {"value": rate, "unit": "updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def member_oracle_leg(wls, runs, nsteps, max_cells):
    """CPU-baseline leg of an ensemble variant: the oracle (as it stands, on
    the host cores) runs each member with at most ``max_cells`` cells from its
    initial state for ``nsteps`` CFL steps, once; ``runs`` maps a name to
    (member states, member times) of ensembles that took the same steps.
    Returns the oracle's rate and, per run, each member's error against it
    (elevation and tracer against max(|oracle|, 1), discharge against the
    oracle's max |q|, the relative difference of the member's time; None for
    members not run) and the worst of them."""
    from oracle.oracle import Oracle
    errs = {k: [] for k in runs}
    cells, t0 = 0, time.perf_counter()
    for m, wl in enumerate(wls):
        if wl.mesh.n > max_cells:
            for k in runs:
                errs[k].append(None)
            continue
        o = Oracle.from_workload(wl)
        to = o.step(nsteps, -1.0, 0.0)
        so = o.get_state()
        cells += wl.mesh.n
        qs = max(float(np.abs(so[1]).max()), float(np.abs(so[2]).max()), 1e-3)
        for k, (states, times) in runs.items():
            st = states[m]
            errs[k].append({
                "zeta": float(np.abs(st[0] - so[0]).max()) / max(float(np.abs(so[0]).max()), 1.0),
                "q": max(float(np.abs(st[i] - so[i]).max()) for i in (1, 2)) / qs,
                "c": float(np.abs(st[3] - so[3]).max()),
                "t_rel": abs(times[m] - to) / to})
    el = time.perf_counter() - t0
    nd = (wls[0].degree + 1) ** 2
    done = sum(1 for e in next(iter(errs.values())) if e is not None)
    leg = {"value": cells * 4 * nd * STAGES * nsteps / el, "unit": "updates/s",
           "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)), "kind": "oracle",
           "sample": f"{done} members with <= {max_cells} cells, {nsteps} CFL steps each, "
                     f"{el:.1f} s"}
    out = {}
    for k, e in errs.items():
        ok = [x for x in e if x is not None]
        out[f"per_member_oracle_err_{k}"] = [
            None if x is None else {a: float(f"{b:.3g}") for a, b in x.items()} for x in e]
        out[f"max_member_oracle_err_{k}"] = (
            {a: max(x[a] for x in ok) for a in ("zeta", "q", "c", "t_rel")} if ok else {})
    return leg, out


def fresh_ensemble_states(wls, stream, nsteps, precision):
    """member states and times of a fresh ensemble after nsteps CFL steps"""
    from paper_2505_18743_gb300 import swdg
    e = swdg.Ensemble.from_workloads(wls, stream=stream.cuda_stream, precision=precision)
    e.step(nsteps)
    tm, _ = e.times()
    st = [e.member_state(m) for m in range(len(wls))]
    e.close()
    return st, list(tm)


def timed_ms(fn, stream, dev, world):
    import torch
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    s0.record(stream)
    fn()
    s1.record(stream)
    torch.cuda.synchronize(dev)
    return max_over_ranks(s0.elapsed_time(s1), world)


def ensemble_small_variant(args, stream, dev, world, members=64, n=32):
    """Many small members, where one launch over all of them should matter:
    64 tidal beaches of 32 x 32 cells each (the ensemble recipe with every
    mesh 32^2: 65 536 cells in all), r = 2, 8 x 8 px per cell, per-member tide
    and Manning n.  FP32-bulk and FP64 ensembles (one CUDA graph per step)
    against the same members as 64 sequential FP64 contexts; the graph's step
    time against the sum of its kernels' times (what a single persistent
    kernel could at most save); and, as the CPU-baseline leg, every member's
    error against the oracle after the same steps."""
    from paper_2505_18743_gb300 import swdg
    wls = W.beach_ensemble(members=members, sizes=(n,))
    nd = (wls[0].degree + 1) ** 2
    cells = sum(w.mesh.n for w in wls)
    units = cells * 4 * nd * STAGES
    steps = max(5, min(args.steps, 20))
    out = {"workload": f"{members} tidal beaches of {n}x{n} cells ({cells} cells), r=2, 8x8 "
                       "px/cell, RK32-IMEX, per-member tide and Manning n", "steps": steps}
    ens = swdg.Ensemble.from_workloads(wls, stream=stream.cuda_stream, precision=1)
    ens.autotune(repeats=1)
    for _ in range(args.warmup):
        ens.step(1)
    ms = timed_ms(lambda: ens.step(steps), stream, dev, world)
    kms, _ = ens.step_profile(steps)
    ksum = sum(kms) / steps
    out["fp32_bulk_ensemble"] = {"value": units * steps * world / (ms / 1e3), "unit": "updates/s",
                                 "ms_per_step": ms / steps,
                                 "kernel_ms_per_step_sum": ksum,
                                 "launches_per_step": 3 * STAGES + 1}
    ens64 = swdg.Ensemble.from_workloads(wls, stream=stream.cuda_stream)
    ens64.autotune(repeats=1)
    for _ in range(args.warmup):
        ens64.step(1)
    ms64 = timed_ms(lambda: ens64.step(steps), stream, dev, world)
    out["fp64_ensemble"] = {"value": units * steps * world / (ms64 / 1e3), "unit": "updates/s",
                            "ms_per_step": ms64 / steps}
    seq = [swdg.Context.from_workload(w, stream=stream.cuda_stream) for w in wls]
    ts = [0.0] * len(seq)
    for i, c in enumerate(seq):
        for _ in range(args.warmup):
            ts[i] = c.step(1, -1.0, ts[i])

    def run_seq():
        for i, c in enumerate(seq):
            ts[i] = c.step(steps, -1.0, ts[i])

    mss = timed_ms(run_seq, stream, dev, world)
    out["fp64_sequential_baseline"] = {"value": units * steps * world / (mss / 1e3),
                                       "unit": "updates/s", "ms_per_step": mss / steps}
    out["speedup_fp64_ensemble_vs_sequential"] = mss / ms64
    out["speedup_fp32_bulk_ensemble_vs_sequential_fp64"] = mss / ms
    for c in seq:
        c.close()
    if not args.no_cpu_baseline:
        k = 8
        runs = {"fp64": fresh_ensemble_states(wls, stream, k, 0),
                "fp32_bulk": fresh_ensemble_states(wls, stream, k, 1)}
        leg, errs = member_oracle_leg(wls, runs, k, n * n)
        out["cpu_baseline"] = leg
        out.update(errs)
    ens.close()
    ens64.close()
    return out


def ensemble_variant(args, stream, dev, world, members=64):
    """A 64-member parameter sweep of tidal beaches (mesh N x N with N drawn
    from 32, 64, 128, 256; r = 2; 8 x 8 px per cell; tide amplitude and
    Manning coefficient drawn per member) in FP32-bulk, every step one
    CUDA-graph launch sequence over all members after the autotuner picked
    the launch shapes; against it the same members as 64 sequential FP64
    contexts and as one FP64 ensemble, and the FP32-bulk members' state error
    against the sequential FP64 runs."""
    import torch
    from paper_2505_18743_gb300 import swdg
    wls = W.beach_ensemble(members=members)
    nd = (wls[0].degree + 1) ** 2
    cells = sum(w.mesh.n for w in wls)
    units = cells * 4 * nd * STAGES
    steps = max(2, min(args.steps, 5))

    def timed(fn):
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        s0.record(stream)
        fn()
        s1.record(stream)
        torch.cuda.synchronize(dev)
        return max_over_ranks(s0.elapsed_time(s1), world)

    out = {"workload": f"{members} tidal beaches, N x N cells with N drawn from 32/64/128/256 "
                       f"({cells} cells in all), r=2, 8x8 px/cell, RK32-IMEX, per-member tide "
                       "and Manning n, each member its own CFL step",
           "cells": cells, "steps": steps}
    ens = swdg.Ensemble.from_workloads(wls, stream=stream.cuda_stream, precision=1)
    tune = ens.autotune(repeats=1)
    for _ in range(args.warmup):
        ens.step(1)
    ms = timed(lambda: ens.step(steps))
    out["fp32_bulk_ensemble"] = {"value": units * steps * world / (ms / 1e3), "unit": "updates/s",
                                 "ms_per_step": ms / steps, "launch_shapes": tune}
    ens64 = swdg.Ensemble.from_workloads(wls, stream=stream.cuda_stream)
    ens64.autotune(repeats=1)
    for _ in range(args.warmup):
        ens64.step(1)
    ms64 = timed(lambda: ens64.step(steps))
    out["fp64_ensemble"] = {"value": units * steps * world / (ms64 / 1e3), "unit": "updates/s",
                            "ms_per_step": ms64 / steps}
    del ens64
    seq = [swdg.Context.from_workload(w, stream=stream.cuda_stream) for w in wls]
    ts = [0.0] * len(seq)
    for i, c in enumerate(seq):
        for _ in range(args.warmup):
            ts[i] = c.step(1, -1.0, ts[i])

    def run_seq():
        for i, c in enumerate(seq):
            ts[i] = c.step(steps, -1.0, ts[i])

    mss = timed(run_seq)
    out["fp64_sequential_baseline"] = {"value": units * steps * world / (mss / 1e3),
                                       "unit": "updates/s", "ms_per_step": mss / steps,
                                       "kind": "64 stand-alone FP64 contexts stepped one after "
                                               "another (each its own CUDA graph)"}
    out["speedup_fp32_bulk_ensemble_vs_sequential_fp64"] = mss / ms
    # FP32-bulk members against the FP64 runs after the same number of steps
    worst = {"zeta": 0.0, "q": 0.0, "c": 0.0}
    for m, c in enumerate(seq):
        a, b = ens.member_state(m), c.get_state()
        qs = max(float(np.abs(b[1]).max()), float(np.abs(b[2]).max()), 1e-3)
        worst["zeta"] = max(worst["zeta"], float(np.abs(a[0] - b[0]).max()) /
                            max(float(np.abs(b[0]).max()), 1.0))
        worst["q"] = max(worst["q"], max(float(np.abs(a[i] - b[i]).max()) for i in (1, 2)) / qs)
        worst["c"] = max(worst["c"], float(np.abs(a[3] - b[3]).max()))
    out["max_rel_member_err_fp32_bulk_vs_fp64"] = worst
    out["steps_compared"] = args.warmup + steps
    if not args.no_cpu_baseline:
        # CPU-baseline leg: the oracle on the members of 32^2 and 64^2 cells
        k = 8
        leg, errs = member_oracle_leg(wls, {"fp32_bulk": fresh_ensemble_states(wls, stream, k, 1)},
                                      k, 64 * 64)
        out["cpu_baseline"] = leg
        out.update(errs)
    for c in seq:
        c.close()
    ens.close()
    return out


def adjoint_variant(args, stream, dev, world, nsteps=200, every=20, ngauges=50):
    """Gauge-misfit gradient (the adjoint case, workloads.gauge_misfit_case):
    a 128 x 128-cell, r = 2 crop of the beach (16 x 16 px per cell, the
    shoreline band included) flooded 0.3 m, 50 seeded gauges in wet cells, a
    truth run with the Manning field perturbed by a smooth +-30 % field;
    loss = sum over 200 CFL steps and the gauges of the squared zeta misfit;
    gradients with respect to the per-cell Manning coefficients and
    bathymetry offsets (and the start state), checkpoint every 20 steps.
    Reported: the forward and backward times against the plain forward (one
    CUDA graph per step), the gradient throughput and the peak device memory."""
    import torch
    from paper_2505_18743_gb300 import adjoint, swdg
    wl, xy, man_true = W.gauge_misfit_case(ngauges=ngauges)
    torch.cuda.synchronize(dev)
    free0, _ = torch.cuda.mem_get_info(dev)
    torch.cuda.reset_peak_memory_stats(dev)
    ctx = swdg.Context.from_workload(wl, stream=stream.cuda_stream)
    nd = (wl.degree + 1) ** 2
    units = wl.mesh.n * 4 * nd * STAGES * nsteps
    mk = lambda a, g: torch.tensor(np.asarray(a, dtype=np.float64), device=dev, requires_grad=g)
    state = [mk(a, False) for a in wl.state()]
    man, delta = mk(wl.manning, True), mk(np.zeros(wl.mesh.n), True)

    def ev():
        return torch.cuda.Event(enable_timing=True)

    with torch.cuda.stream(stream):
        with torch.no_grad():
            *_, G_true = adjoint.solve(ctx, *state, mk(man_true, False), delta, nsteps=nsteps,
                                       gauges=xy, checkpoint_every=every)
        # untimed warm-up of the whole path, torch's own loss and autograd kernels
        # included (their first use in a process loads them)
        *_, Gw = adjoint.solve(ctx, *state, man, delta, nsteps=2, gauges=xy, checkpoint_every=every)
        ((Gw - G_true[:2]) ** 2).sum().backward()
        man.grad, delta.grad = None, None
        s0, s1, s2 = ev(), ev(), ev()
        torch.cuda.synchronize(dev)
        s0.record(stream)
        *_, G = adjoint.solve(ctx, *state, man, delta, nsteps=nsteps, gauges=xy,
                              checkpoint_every=every)
        loss = ((G - G_true) ** 2).sum()
        s1.record(stream)
        loss.backward()
        s2.record(stream)
        torch.cuda.synchronize(dev)
    t_fwd, t_bwd = s0.elapsed_time(s1), s1.elapsed_time(s2)
    # the context's buffers persist and torch's caching allocator keeps its
    # reserve, so what is in use now plus what torch gave back is the peak
    free1, _ = torch.cuda.mem_get_info(dev)
    peak_mb = (free0 - free1 + torch.cuda.max_memory_reserved(dev)
               - torch.cuda.memory_reserved(dev)) / 2 ** 20
    torch_mb = torch.cuda.max_memory_allocated(dev) / 2 ** 20
    plain = swdg.Context.from_workload(wl, stream=stream.cuda_stream)
    plain.step(2, -1.0, 0.0)
    plain.set_state(*wl.state())
    p0, p1 = ev(), ev()
    torch.cuda.synchronize(dev)
    p0.record(stream)
    plain.step(nsteps, -1.0, 0.0)
    p1.record(stream)
    torch.cuda.synchronize(dev)
    t_plain = p0.elapsed_time(p1)
    ok = all(bool(torch.isfinite(g).all()) for g in (man.grad, delta.grad))
    out = {"workload": "tidal beach crop 128x128 cells (cells 128..255 x 64..191), r=2, 16x16 "
                       "px/cell (f64), RK32-IMEX, 0.3 m flood, 50 gauges, truth Manning +-30 %",
           "steps": nsteps, "checkpoint_every": every, "loss": float(loss.detach()),
           "forward_ms": t_fwd, "backward_ms": t_bwd, "plain_forward_ms": t_plain,
           "backward_over_plain_forward": t_bwd / t_plain,
           "gradient_updates_per_s": units * world / (t_bwd / 1e3), "unit": "updates/s",
           "device_memory_peak_mb": peak_mb, "torch_tensors_peak_mb": torch_mb,
           "grad_manning_max": float(man.grad.abs().max()),
           "grad_delta_max": float(delta.grad.abs().max()), "gradients_finite": ok}
    ctx.close()
    plain.close()
    return out


def long_run_variant(args, stream, dev, world, chunks=10, chunk=100):
    """The tidal beach's whole 1000-step run (from its initial state at
    t = 0), timed in chunks of 100 steps with CUDA events: the per-step cost
    over the run, and the water-mass balance and wet-dry state at its end."""
    import torch
    from paper_2505_18743_gb300 import swdg
    wl = W.tidal_beach()
    ctx = swdg.Context.from_workload(wl, stream=stream.cuda_stream)
    d0 = ctx.diagnostics()
    t = 0.0
    per = []
    for _ in range(chunks):
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        s0.record(stream)
        t = ctx.step(chunk, -1.0, t)
        s1.record(stream)
        torch.cuda.synchronize(dev)
        per.append(max_over_ranks(s0.elapsed_time(s1), world) / chunk)
    d1 = ctx.diagnostics()
    ctx.close()
    return {"workload": WORKLOAD + f", steps 1..{chunks * chunk} from t = 0",
            "ms_per_step_by_chunk_of_100": [round(x, 4) for x in per],
            "spread": (max(per) - min(per)) / min(per), "t_end_s": t,
            "r_cells_start_end": [d0["r_cells"], d1["r_cells"]],
            "positivity_violations": d1["positivity_violations"]}


def lagoon_static_variant(args, stream, dev, world):
    """The lagoon as a static 2:1 forest (3 levels toward the fractal
    coastline, about 200k cells, r = 2, 32/16/8 px per cell side from one
    8192 x 4096 f32 raster, tide at the south boundary, Manning n = 0.02),
    FP64: hanging-face fluxes and mass across refinement levels.  Timed steps
    with CUDA events, per-kernel times, and the water-mass change over them."""
    import torch
    from paper_2505_18743_gb300 import swdg
    wl = W.lagoon()
    Xn, Yn = W.nodal_coordinates(wl.mesh, wl.degree)
    wl.c = 0.5 + 0.5 * np.tanh((Xn - 25000.0) / 2000.0)
    ctx = swdg.Context.from_workload(wl, stream=stream.cuda_stream)
    nd = (wl.degree + 1) ** 2
    hanging = int((wl.mesh.nbr[:, :, 1] >= 0).sum())
    t = 0.0
    for _ in range(args.warmup):
        t = ctx.step(1, -1.0, t)
    steps = max(5, min(args.steps, 50))
    torch.cuda.synchronize(dev)
    d0 = ctx.diagnostics()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    t = ctx.step(steps, -1.0, t)
    s1.record(stream)
    torch.cuda.synchronize(dev)
    ms = max_over_ranks(s0.elapsed_time(s1), world)
    d1 = ctx.diagnostics()
    kms, t = ctx.step_profile(3, -1.0, t)
    per = {SLOTS[i]: round(kms[i] / 3, 4) for i in range(len(SLOTS)) if kms[i] > 0}
    ctx.close()
    units = wl.mesh.n * 4 * nd * STAGES
    return {"workload": f"lagoon 50x30 km, static 2:1 forest, 3 levels ({wl.mesh.n} cells, "
                        f"{hanging} hanging face slots), r=2, 32/16/8 px per cell, tide at the "
                        "south, Manning 0.02, RK32-IMEX, FP64",
            "cells": wl.mesh.n, "steps": steps, "ms_per_step": ms / steps,
            "value": units * steps * world / (ms / 1e3), "unit": "updates/s",
            "per_launch_ms": per,
            "water_mass_change_rel_with_tide": abs(d1["mass"] - d0["mass"]) / d0["mass"],
            "positivity_violations": d1["positivity_violations"]}


def amr_variant(args, stream, dev, world, cycles=4, every=5):
    """Dynamic h-adaptation on the lagoon (256 x 128 coarse cells of
    195 x 234 m, up to two refinements (three levels), r = 2, 8192 x 4096 f32 raster, tide
    on the south): every 5 steps the |grad c| indicator (Sec. 5), the
    criteria of Sec. 3.4 (theta_r = 0.3, theta_c = 0.05), the forest
    adaptation, the remap and the re-upload; the share of the adaptation in
    the wall time and the accumulated |Q^n| relative to the initial mass."""
    import torch
    from paper_2505_18743_gb300 import swdg
    wl = W.lagoon()
    Xn, Yn = W.nodal_coordinates(wl.mesh, wl.degree)
    wl.c = 0.5 + 0.5 * np.tanh((Xn - 25000.0) / 2000.0)  # a tracer front across the lagoon
    ctx = swdg.Context.from_workload(wl, stream=stream.cuda_stream)
    ctx.amr_setup(swdg.make_forest(256, 128, 0.0, 0.0, 50000.0 / 256, 30000.0 / 128, 2, 0.0,
                                   (0, 0, 1, 0), (False, False)))
    h0 = ctx.diagnostics()["mass"]
    t = 0.0
    t = ctx.step(2, -1.0, t)  # warm-up
    step_ms, adapt_ms, cells, qsum, split = [], [], [wl.mesh.n], 0.0, []
    for _ in range(cycles):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        t = ctx.step(every, -1.0, t)
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        rep = ctx.amr_adapt(0.3, 0.05, kind=1)
        torch.cuda.synchronize(dev)
        t2 = time.perf_counter()
        step_ms.append(1e3 * (t1 - t0) / every)
        adapt_ms.append(1e3 * (t2 - t1))
        split.append([round(rep[k], 2) for k in ("indicator_ms", "forest_ms", "rebuild_ms")])
        cells.append(int(rep["cells_after"]))
        qsum += abs(rep["Q"])
    ctx.close()
    steps_total = sum(step_ms) * every
    return {"workload": "lagoon 256x128 coarse cells, 2 levels, r=2, |grad c| indicator, "
                        "adaptation every 5 steps",
            "cells": cells, "step_ms": [round(x, 3) for x in step_ms],
            # DoF-stage updates/s of the steps of each cycle (on that cycle's mesh)
            "updates_per_s": [cells[i] * 4 * (wl.degree + 1) ** 2 * STAGES / (step_ms[i] / 1e3)
                              for i in range(len(step_ms))],
            "adapt_ms": [round(x, 2) for x in adapt_ms],
            "adapt_split_ms_indicator_forest_rebuild": split,
            "adaptation_share_of_wall_time": sum(adapt_ms) / (steps_total + sum(adapt_ms)),
            "sum_abs_Q_over_initial_mass": qsum / h0}


def run_gpu(args, rank, world, local):
    import torch
    from paper_2505_18743_gb300 import swdg
    dev = torch.device("cuda", local)
    wl = W.tidal_beach()
    stream = torch.cuda.Stream(device=dev)
    prec = 1 if args.precision == "fp32bulk" else 0
    ctx = swdg.Context.from_workload(wl, stream=stream.cuda_stream, precision=prec)
    units = units_per_step(wl)
    t = 0.0
    # warm-up (also captures the step graph)
    for _ in range(args.warmup):
        t = ctx.step(1, -1.0, t)
    torch.cuda.synchronize(dev)
    barrier(world)
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize(dev)
        barrier(world)
        start.record(stream)
        t = ctx.step(args.steps, -1.0, t)
        end.record(stream)
        torch.cuda.synchronize(dev)
        barrier(world)
    ms = start.elapsed_time(end)
    ms = max_over_ranks(ms, world)
    value = units * args.steps * world / (ms / 1e3)
    clocks = clk.summary()

    # per-kernel durations (CUDA events on the context's stream, eager launches)
    kms, t = ctx.step_profile(max(2, min(args.steps, 5)), -1.0, t)
    nprof = max(2, min(args.steps, 5))
    per_launch = {SLOTS[i]: kms[i] / nprof for i in range(len(SLOTS)) if kms[i] > 0}
    total = sum(per_launch.values())
    # the dominant kernel: the kernel function with the largest share of the step
    fn_of = lambda k: ("k_residual" if k.startswith("residual") else "k_faces" if
                       k.startswith("faces") else "k_stage" if (k.startswith("stage") or
                                                                k == "final") else "k_step_begin")
    share = {}
    for k, v in per_launch.items():
        share[fn_of(k)] = share.get(fn_of(k), 0.0) + v
    dom_fn = max(share, key=share.get)
    slots = [k for k in per_launch if fn_of(k) == dom_fn]
    avg_ms = sum(per_launch[k] for k in slots) / len(slots)
    counters, fresh = load_counters()
    table = counters["fp64" if prec == 0 else "fp32bulk"]
    flops = sum(table[k][0] for k in slots) / len(slots) * wl.mesh.n
    ach = flops / (avg_ms / 1e3) / 1e12
    pk, src = peaks()
    nres = {"stage_2": 1, "stage_3": 2, "stage_4": 3, "final": STAGES}
    bpc = sum(algorithmic_bytes_per_cell(k, nres=nres.get(k, STAGES)) for k in slots) / len(slots)
    hbm_ach = bpc * wl.mesh.n / (avg_ms / 1e3) / 1e9
    # DRAM bytes per launch from the ncu capture, only while it matches the kernels
    traffic = [table[k][2] if fresh else None for k in slots]
    pipe = measured_pipe_peaks()
    if "fp64" in pipe:
        fp64_peak = pipe["fp64"][0]
        peak_src = ("FP64 pipe, measured in this run by the FMA-chain probe (swdg_probe_fma), "
                    "of measured")
    else:
        fp64_peak = FP64_PEAK_TFLOPS
        peak_src = "FP64 pipe, nominal 152 SMs x 2.07 GHz x 4 flop/clk (probe unavailable)"
    roof = {"bound": "alu", "kernel": dom_fn, "achieved": ach, "peak": fp64_peak,
            "unit": "TFLOP/s", "frac": ach / fp64_peak,
            "traffic": (sum(traffic) / len(traffic)) if all(x is not None for x in traffic) else None,
            "peak_source": peak_src,
            "pipe_peaks_measured_tflops": {k: round(v[0], 3) for k, v in pipe.items()},
            "counters": "profiles/counters_tidal_beach_256x256_r3.txt" + ("" if fresh else
                                                                         " (stale: kernels changed)"),
            "flops_per_launch": flops, "avg_launch_ms": avg_ms, "share": share[dom_fn] / total,
            "hbm_view": {"achieved_gbs": hbm_ach, "peak_gbs": pk["hbm_gbs"],
                         "frac": hbm_ach / pk["hbm_gbs"], "peak_source": src},
            "per_launch_ms": {k: round(v, 4) for k, v in per_launch.items()}}

    # end to end: host state in, one step, host state out, every step
    nd = (wl.degree + 1) ** 2
    host = [torch.empty((wl.mesh.n, nd), dtype=torch.float64).pin_memory() for _ in range(4)]
    ctx.get_state(host)
    e2e_steps = max(1, min(args.steps, 5))
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ctx.set_state(*host)
        t = ctx.step(1, -1.0, t)
        ctx.get_state(host)
    el = time.perf_counter() - t0
    el = max_over_ranks(el, world)
    bytes_io = 4 * wl.mesh.n * nd * 8
    e2e = {"value": units * e2e_steps * world / el, "unit": "updates/s",
           "h2d_bytes_per_step": bytes_io, "d2h_bytes_per_step": bytes_io}

    # FP32-bulk variant on the same workload: same timing, plus its state error
    # against this FP64 run after the same steps from the same initial state
    variants = {}
    want = set() if args.no_variants else set(args.variants.split(","))
    if "fp32_bulk" in want and prec == 0:
        ref_state = ctx.get_state()
        t_ref = t
        ctx32 = swdg.Context.from_workload(wl, stream=stream.cuda_stream, precision=1)
        t32 = 0.0
        for _ in range(args.warmup):
            t32 = ctx32.step(1, -1.0, t32)
        torch.cuda.synchronize(dev)
        s32, e32 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s32.record(stream)
        t32 = ctx32.step(args.steps, -1.0, t32)
        e32.record(stream)
        torch.cuda.synchronize(dev)
        ms32 = max_over_ranks(s32.elapsed_time(e32), world)
        # replay the FP64 context's extra profile/e2e steps so both reach the same
        # step count: the profiled steps (kernels launched one by one, timed each)
        # and the rest as plain steps
        kms32, t32 = ctx32.step_profile(nprof, -1.0, t32)
        per32 = {SLOTS[i]: round(kms32[i] / nprof, 4) for i in range(len(SLOTS)) if kms32[i] > 0}
        extra = nprof + e2e_steps
        t32 = ctx32.step(e2e_steps, -1.0, t32)
        st32 = ctx32.get_state()
        errs = {}
        qscale = max(float(np.abs(ref_state[1]).max()), float(np.abs(ref_state[2]).max()), 1e-3)
        for name, a, b in zip(("zeta", "qx", "qy", "c"), st32, ref_state):
            # elevation and tracer against their O(1) scale, discharges against |q|max
            den = max(float(np.abs(b).max()), 1.0) if name in ("zeta", "c") else qscale
            errs[name] = float(np.abs(a - b).max()) / den
        d64, d32 = ctx.diagnostics(), ctx32.diagnostics()
        variants["fp32_bulk"] = {
            "value": units * args.steps * world / (ms32 / 1e3), "unit": "updates/s",
            "ms_per_step": ms32 / args.steps, "dtype": "f64 elevation/sub-grid/solves, f32 bulk",
            "per_launch_ms": per32,
            "max_rel_state_err_vs_fp64": errs,
            "steps_compared": args.warmup + args.steps + extra,
            "mass_rel_diff_vs_fp64": abs(d32["mass"] - d64["mass"]) / d64["mass"],
            "time_matches": abs(t32 - t_ref) <= 1e-9 * max(t_ref, 1.0)}
        ctx32.close()

    if prec == 0:
        for name, fn in (("long_run", long_run_variant), ("ensemble", ensemble_variant),
                         ("ensemble_small", ensemble_small_variant),
                         ("lagoon_static", lagoon_static_variant),
                         ("adjoint", adjoint_variant), ("amr", amr_variant)):
            if name in want:
                variants[name] = fn(args, stream, dev, world)

    line = {"metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == 0 else "f64 elevation/sub-grid/solves, f32 bulk",
            "data": "synthetic",
            "config": {"workload": WORKLOAD if prec == 0 else WORKLOAD.replace("FP64", "FP32-bulk"), "cells": wl.mesh.n, "degree": wl.degree,
                       "pixels_per_cell": 256, "stages": STAGES,
                       "l2": "inputs larger than L2 (about 0.5 GB working set), no flush",
                       "parallelism": f"replicas x{world}"},
            "clocks": clocks, "roofline": roof, "e2e": e2e, "variants": variants,
            # per step: step_begin, per stage k_faces + k_residual, the stage
            # updates and the final combination (3 STAGES + 1); plus the clock
            # upload of the step call
            "gpu_launches": (3 * STAGES + 1) * args.steps + 1}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, cores, sample = cpu_oracle_rate()
        line["cpu_baseline"] = {"value": rate, "unit": "updates/s", "cores": cores,
                                "kind": "oracle", "sample": sample}
        # the same oracle on one thread (a shorter sample)
        if omp_threads(1):
            r1, _, s1 = cpu_oracle_rate(seconds=5.0)
            omp_threads(cores)
            line["cpu_baseline"]["single_thread"] = {"value": r1, "unit": "updates/s",
                                                     "cores": 1, "sample": s1}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="swdg", choices=["swdg", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--variants",
                    default="fp32_bulk,long_run,ensemble,ensemble_small,lagoon_static,adjoint,amr",
                    help="comma-separated variants to run after the headline line")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32bulk"],
                    help="arithmetic of the timed context (fp64 is the headline workload)")
    args = ap.parse_args()
    rank, world, local = dist_init(args.gpus)
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_gpu(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
