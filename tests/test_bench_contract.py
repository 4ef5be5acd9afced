"""bench.py's command-line contract on the CPU, through its reference arm (the
CPU oracle timed on the host cores, which needs no GPU): one JSON line with
the primary line's metric, unit and direction, the reference keys
(impl, cpu_baseline, e2e with no host-device bytes), and, for N > 1, one line
printed by rank 0 alone -- both when torchrun launches the ranks and when
bench.py, started with --gpus N and no WORLD_SIZE, relaunches itself under
torchrun.  The oracle sample is one 1600-cell profile, a few steps."""
import json
import os
import socket
import subprocess
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
BENCH = str(ROOT / "bench.py")
METRIC = "TENO7 RK3 Gcell-updates/s (1D Euler, tiled Shu-Osher)"


def _run(cmd):
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK", "MASTER_PORT")}
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    return json.loads(lines[0])


def _check_reference_line(d, world, steps, warmup):
    assert d["impl"] == "reference" and d["metric"] == METRIC and d["unit"] == "Gcell-steps/s"
    assert d["higher_is_better"] is True and d["vs_baseline"] is None and d["data"] == "synthetic"
    assert d["n_gpus"] == world and d["steps"] == steps and d["warmup"] == max(warmup, 3)
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert "N=1600 cells" in d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_one_process():
    d = _run([sys.executable, BENCH, "--impl", "reference", "--steps", "2", "--warmup", "0", "--ref-tiles", "1"])
    _check_reference_line(d, 1, 2, 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_reference_arm_under_torchrun_prints_once():
    d = _run([sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2",
              "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), BENCH, "--impl", "reference",
              "--gpus", "2", "--steps", "1", "--warmup", "3", "--ref-tiles", "1"])
    _check_reference_line(d, 2, 1, 3)


def test_bench_relaunches_itself_for_several_gpus():
    d = _run([sys.executable, BENCH, "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3",
              "--ref-tiles", "1"])
    _check_reference_line(d, 2, 1, 3)
