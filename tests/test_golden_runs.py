"""The stored whole-run hashes (golden/runs_f64.txt) are the rows that
golden/make_runs.py lists -- same names, systems, sizes and step counts -- and
well formed, so that the GPU tests that read them compare against the runs
the script describes.  (Recomputing the hashes takes the oracle 5 to 15
minutes per run: python tests/golden/make_runs.py.)"""
import importlib.util
import math
from pathlib import Path

import oracle_runs

GOLDEN = Path(__file__).parent / "golden"


def _script():
    spec = importlib.util.spec_from_file_location("make_runs", GOLDEN / "make_runs.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_stored_runs_are_the_scripts():
    want = {r[0]: r[1:] for r in _script().RUNS}
    got = {}
    for system in ("euler1d", "euler2d"):
        for name, seed, nx, ny, steps, t_end, digest in oracle_runs.rows(system):
            got[name] = (system, seed, nx, ny, steps)
            assert math.isfinite(t_end) and t_end > 0.0
            assert len(digest) == 64 and int(digest, 16) >= 0
    assert got == want
