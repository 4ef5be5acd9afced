"""The index-checked build (libteno7_checked.so, compiled with T7_CHECKED=1 --
the stand-in for a memory checker): every cell, row and column index the
kernels form for a global-memory access is tested against the extent of its
array, and a failing one returns T7_EINDEX.  checked_driver.py takes every
form of the forward path through the C ABI at ragged and tiny sizes: 1D
advection, Burgers and Euler in FP64, FP32 and mixed precision with both
schemes (N = 3, 61, 97, 122, 200, 759), host-array runs with the parted last
stage, per-field alphas, the discrete adjoint (RHS, step, recorded step) and
the no-allocation step, slabs of one domain, a ragged batch with tubes of 3
to 1000 cells and two group sizes; 2D in every precision at 5 x 7 to
200 x 233, periodic and transmissive, whole and in slabs.  With the checked
build it must finish without any error status; its FP64 results equal the
release build's bit for bit, and the FP32 and mixed ones agree within FP32
rounding (the checks add control flow, around which the compiler may contract
an FP32 multiply-add differently).  The adjoint's outputs, summed by atomic
adds in an order that varies from run to run, agree within FP64 (FP32)
rounding."""
import os
import subprocess
import sys
from pathlib import Path

import numpy as np
import pytest

from paper_1808_00037_gb300 import build

pytestmark = pytest.mark.gpu

ROOT = Path(__file__).resolve().parents[1]


def _drive(lib, out):
    env = dict(os.environ, T7_LIBRARY=str(lib))
    r = subprocess.run([sys.executable, str(ROOT / "tests" / "checked_driver.py"), str(out)], env=env,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-4000:]
    with np.load(out) as z:
        return {k: z[k] for k in z.files}


def test_checked_build_runs_every_form_and_agrees(tmp_path):
    release = build.build()
    checked = build.build(checked=True)
    rel = _drive(release, tmp_path / "release.npz")
    chk = _drive(checked, tmp_path / "checked.npz")
    assert rel.keys() == chk.keys() and len(rel) > 150
    for k, a in rel.items():
        b = chk[k]
        assert a.shape == b.shape and a.dtype == b.dtype, k
        scattered = k.startswith("adj-") and k.rsplit("-", 1)[1] in ("rhs", "step", "recorded")
        if scattered:
            # the adjoint scatters with atomic adds: its bits follow their order
            tol = 1e-12 if "f64" in k else 1e-4
            assert np.abs(a - b).max() <= tol * max(np.abs(a).max(), 1e-300), k
        elif "f64" in k or k.endswith("-steps"):
            assert np.array_equal(a, b), k
        elif a.dtype == np.uint8:  # Delta codes
            assert (a == b).mean() >= 0.999, k
        else:
            scale = max(np.abs(a).max(), 1e-30)
            assert np.abs(a - b).max() <= 1e-4 * scale, (k, np.abs(a - b).max(), scale)


@pytest.mark.parametrize("i,lo,hi", [(5, 0, 10), (0, 0, 10), (9, 0, 10), (10, 0, 10), (-1, 0, 10),
                                     (-4, -4, 20), (-5, -4, 20), (20, -4, 20), (123456, 0, 100)])
def test_index_check_latches_and_clamps(i, lo, hi):
    """The check itself (t7_probe_index_check, one index through it on a
    private control block): in the checked build an index outside [lo, hi)
    is latched with its value and replaced by lo, one inside passes
    unchanged; the release build passes every index unchanged and latches
    nothing."""
    from paper_1808_00037_gb300 import binding as B
    inside = lo <= i < hi
    idx, flagged, checked = B.probe_index_check(i, lo, hi, lib=B.load(build.build(checked=True)))
    assert checked and idx == (i if inside else lo) and flagged == (not inside)
    idx, flagged, checked = B.probe_index_check(i, lo, hi, lib=B.load(build.build()))
    assert not checked and idx == i and not flagged
