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
