"""The JSON line of `bench.py --impl reference` (the oracle timed on the host
cores): its keys and values, alone and under torchrun with two ranks on the
gloo backend, where rank 0 alone runs and prints and the other rank exits 0
without work.  CPU only."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lines(out):
    return [json.loads(l) for l in out.splitlines() if l.startswith("{")]


def _check_line(r, n_gpus, steps, warmup):
    assert r["impl"] == "reference"
    assert r["metric"] == "DoF-stage updates/s" and r["unit"] == "updates/s"
    assert r["higher_is_better"] is True and r["n_gpus"] == n_gpus
    assert r["steps"] == steps and r["warmup"] == warmup
    assert r["value"] > 0 and r["ms_per_step"] > 0
    assert r["dtype"] == "f64" and r["data"] == "synthetic" and r["vs_baseline"] is None
    assert "workload" in r["config"]
    cb = r["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == r["value"] and cb["cores"] >= 1
    assert cb["sample"]
    e2e = r["e2e"]
    assert e2e == {"value": r["value"], "unit": r["unit"], "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}


def test_reference_arm_prints_one_contract_line():
    p = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = _lines(p.stdout)
    assert len(lines) == 1
    _check_line(lines[0], 1, 1, 3)


def test_reference_arm_under_two_gloo_ranks_prints_once():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    p = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                        "--nproc-per-node", "2", "--master-addr", "127.0.0.1",
                        "--master-port", str(port), "bench.py", "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = _lines(p.stdout)
    assert len(lines) == 1
    _check_line(lines[0], 2, 1, 3)


def _bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def test_clock_summary_reports_median_max_and_throttle_reasons(tmp_path):
    bench = _bench()
    rows = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 1200.5, 0x0, Not Active, Not Active, Not Active, Not Active",
            "bad line"]
    p = tmp_path / "clocks.csv"
    p.write_text("\n".join(rows) + "\n")
    s = bench.ClockSampler()
    s.path = str(p)
    out = s.summary()
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                   "samples": 3}
    # every throttle reason the timing rules name is reported
    p.write_text("0, 1500, 2070, 1000, 0x68, Active, Active, Active, Not Active\n")
    s.path = str(p)
    assert s.summary()["reasons"] == ["hw_slowdown", "hw_thermal_slowdown",
                                      "sw_thermal_slowdown"]
    # no samples at all: said so, not left empty
    s.path = str(tmp_path / "missing.csv")
    assert s.summary()["reasons"] == ["unavailable"]


def test_algorithmic_bytes_match_the_per_cell_model():
    """r = 3, 16 x 16 f32 pixels per cell: residual 4 + 6 fields of 16 f64
    nodes, the 1 KB tile and 57 B of geometry; stage update v^n, H and C~,
    nres residual sets of 6 fields and the output state."""
    b = _bench().algorithmic_bytes_per_cell
    assert b("residual_2") == 4 * 16 * 8 + 6 * 16 * 8 + 16 * 16 * 4 + 57 == 2361
    assert b("stage_2", nres=1) == 2121 and b("final", nres=3) == 3657
    assert b("step_begin") == 1865 and b("faces_1") == 4 * 16 * 8 + 57
    assert _bench().units_per_step(type("W", (), {"degree": 3, "mesh": type(
        "M", (), {"n": 65536})})()) == 65536 * 4 * 16 * 3


def _max_worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), CUDA_VISIBLE_DEVICES="")
    sys.path.insert(0, ROOT)
    import bench
    r, w, _ = bench.dist_init(world)
    assert (r, w) == (rank, world)
    bench.barrier(w)
    # each rank's timed region; the job's time is the slowest rank's
    out[rank] = bench.max_over_ranks(10.0 + 5.0 * rank, w)
    bench.barrier(w)
    dist.destroy_process_group()


def test_max_over_ranks_takes_the_slowest_of_two_gloo_ranks():
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_max_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=300)
            assert p.exitcode == 0
        assert dict(out) == {0: 15.0, 1: 15.0}


def test_counters_profile_covers_every_launch_slot():
    """bench.py takes its roofline flops and DRAM traffic from the committed
    ncu summary: every launch slot of a step, both precisions, with the
    hash of the kernel sources it was taken on"""
    import bench
    table, _ = bench.load_counters()
    slots = {"step_begin", "faces_1", "faces_2", "faces_3", "residual_1", "residual_2",
             "residual_3", "stage_2", "stage_3", "final"}
    for prec in ("fp64", "fp32bulk"):
        assert set(table[prec]) == slots
        for f64, f32, dram in table[prec].values():
            assert f64 > 0 and dram > 0
    h = bench.kernel_sources_hash()
    assert len(h) == 16 and h == bench.kernel_sources_hash()
