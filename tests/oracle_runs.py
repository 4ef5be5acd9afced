"""Reader of golden/runs_f64.txt: whole FP64 oracle runs on the benchmark
workloads (written by golden/make_runs.py, which calls the oracle only),
stored as step count, end time and a SHA-256 of the end state."""
import hashlib
from pathlib import Path

import numpy as np

PATH = Path(__file__).parent / "golden" / "runs_f64.txt"


def rows(system):
    """(name, seed-or-tiles, nx, ny, steps, t_end, sha256) of every stored run
    of one system ("euler1d" or "euler2d")."""
    out = []
    for line in PATH.read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            name, sysname, seed, nx, ny, steps, t, digest = line.split()
            if sysname == system:
                out.append((name, int(seed), int(nx), int(ny), int(steps), float.fromhex(t), digest))
    return out


def state_hash(U):
    """SHA-256 of the float64 little-endian bytes of U in C order."""
    return hashlib.sha256(np.ascontiguousarray(U, dtype="<f8").tobytes()).hexdigest()
