"""Writes runs_f64.txt: whole FP64 runs of the CPU oracle on the benchmark
workloads, stored as step count, end time and a SHA-256 of the end state, for
runs too long to repeat inside a test (5 to 15 minutes each on one host core).

Rows (SSP-RK3 steps of Sec. 2.1 with the CFL step of the global
Lax-Friedrichs alpha, Sec. "One dimensional Euler equations"; gamma 1.4,
C_T = 1e-5, epsilon = dx^3):
  - 1D Euler, the Shu-Osher profile (inputs.shu_osher: 1600 cells on [-5, 5])
    tiled 10486 times to 16,777,600 cells, zero-gradient ends, CFL 0.5;
  - 2D Euler, four-quadrant Riemann data (inputs.quadrants_2d(seed, nx, ny)),
    zero-gradient on all four sides, CFL 0.4, dimension by dimension: 256^2
    for 500 steps and the full 2048^2 for 20.
The hash is over the float64 bytes of U ([3][n] or [4][ny][nx], C order, little
endian).  The oracle evaluates + - * / and sqrt only, compiled without
contraction, so the stored bits do not depend on the host.

Run from the repository root:  python tests/golden/make_runs.py
"""
import hashlib
import math
import multiprocessing as mp
import sys
from concurrent.futures import ProcessPoolExecutor
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

import oracle  # noqa: E402
from paper_1808_00037_gb300 import inputs as I  # noqa: E402

# (name, system, seed or tiles, nx, ny, steps)
RUNS = (
    ("quadrants-256-500", "euler2d", 2024, 256, 256, 500),
    ("quadrants-2048-20", "euler2d", 2024, 2048, 2048, 20),
    ("shu-osher-x10486-20", "euler1d", 10486, 1600 * 10486, 1, 20),
)
OUT = Path(__file__).with_name("runs_f64.txt")


def state_hash(U):
    return hashlib.sha256(np.ascontiguousarray(U, dtype="<f8").tobytes()).hexdigest()


def run(name, system, seed, nx, ny, steps):
    if system == "euler2d":
        U, dx, dy, _ = I.quadrants_2d(seed, nx, ny)
        Uo, so, to, st = oracle.run_2d(U, dx, dy, cfl=0.4, max_steps=steps)
    else:
        U, dx = I.shu_osher(1600, tiles=seed)
        assert U.shape[1] == nx
        Uo, so, to, st = oracle.run_1d(oracle.SYS_EULER1D, U, dx, t_end=math.inf, cfl=0.5, bc=(1, 1),
                                       max_steps=steps)
    assert st == 0 and so == steps, (name, st, so)
    line = f"{name} {system} {seed} {nx} {ny} {so} {float(to).hex()} {state_hash(Uo)}"
    print(line, flush=True)
    return line


def main():
    lines = ["# FP64 oracle runs on the benchmark workloads; written by tests/golden/make_runs.py (calls the",
             "# oracle only).  Columns: name system seed-or-tiles nx ny steps t_end(hex) sha256(U, float64 LE)"]
    # one process per run (the runs are independent)
    with ProcessPoolExecutor(len(RUNS), mp_context=mp.get_context("spawn")) as ex:
        lines += list(ex.map(run, *zip(*RUNS)))
    OUT.write_text("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
