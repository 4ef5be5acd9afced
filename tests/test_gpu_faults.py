"""Fault injection on the host: poisoned states (NaN, Inf, a negative density,
a negative pressure) handed to the forward entry points in every precision,
for 1D, 2D and a ragged batch.  Every call returns the status the header
gives for the fault -- T7_ENONFINITE for Inf/NaN, T7_ENONPHYSICAL for a
finite state with rho <= 0 or p <= 0 -- names a flat cell index next to the
poisoned cell, and leaves the context usable: the next call on a clean state
succeeds.  No GPU fault is involved: the kernels latch a flag and carry on,
and the status comes back from the next synchronising call."""
import re

import numpy as np
import pytest

from paper_1808_00037_gb300 import binding as B
from paper_1808_00037_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

PRECS = [(B.T7_F64, torch.float64), (B.T7_F32, torch.float32), (B.T7_MIXED, torch.float64)]
PREC_IDS = ["f64", "f32", "mixed"]


def poison(U, kind, flat):
    """Poison cell `flat` (flat index over the spatial dimensions) of a
    conserved state U[m, ...] (rho, momenta, E); returns the expected status."""
    V = U.reshape(U.shape[0], -1)
    if kind == "nan_momentum":
        V[1, flat] = np.nan
        return B.T7_ENONFINITE
    if kind == "inf_density":
        V[0, flat] = np.inf
        return B.T7_ENONFINITE
    if kind == "negative_density":
        V[0, flat] = -0.5
        return B.T7_ENONPHYSICAL
    if kind == "negative_pressure":
        V[-1, flat] = -1.0
        return B.T7_ENONPHYSICAL
    raise ValueError(kind)


KINDS = ["nan_momentum", "inf_density", "negative_density", "negative_pressure"]


def reported_index(err):
    m = re.search(r"index (-?\d+)", str(err))
    assert m, str(err)
    return int(m.group(1))


@pytest.mark.parametrize("prec,dtype", PRECS, ids=PREC_IDS)
@pytest.mark.parametrize("kind", KINDS)
def test_1d_poisoned_state_reported_by_every_entry_point(prec, dtype, kind):
    U0, dx = I.shu_osher(1600)
    k = 800
    U = U0.copy()
    want = poison(U, kind, k)
    c = B.Context(B.T7_EULER1D, 1600, dx, prec=prec, bc=(1, 1, 0, 0))

    def dev(A):
        return torch.tensor(A, dtype=dtype, device="cuda")

    calls = {
        "run": lambda: c.run(dev(U), 0.5, max_steps=2),
        "rk3_step": lambda: (c.rk3_step(dev(U), 1e-4), c.sync()),
        "euler_rhs": lambda: (c.euler_rhs(dev(U)), c.sync()),
        "cfl_dt": lambda: c.cfl_dt(dev(U), 0.5),
    }
    for name, call in calls.items():
        with pytest.raises(B.T7Error) as ei:
            call()
        assert ei.value.status == want, (name, str(ei.value))
        # the lowest flagged index: the cell itself, a face next to it, or a
        # cell the stencil reached within the steps taken
        assert k - 30 <= reported_index(ei.value) <= k + 1, (name, str(ei.value))
        # the context stays usable
        steps, _ = c.run(dev(U0), 0.5, max_steps=2)
        assert steps == 2, name


@pytest.mark.parametrize("prec,dtype", PRECS, ids=PREC_IDS)
@pytest.mark.parametrize("kind", KINDS)
def test_2d_poisoned_state_reported(prec, dtype, kind):
    nx, ny = 96, 64
    U0, dx, dy, _ = I.quadrants_2d(4, nx, ny)
    y, x = 40, 50
    U = U0.copy()
    want = poison(U, kind, y * nx + x)
    zg = (B.T7_BC_ZERO_GRADIENT,) * 4
    c = B.Context(B.T7_EULER2D, nx, dx, ny=ny, dy=dy, prec=prec, bc=zg)

    def dev(A):
        return torch.tensor(A, dtype=dtype, device="cuda")

    for name, call in {"run": lambda: c.run(dev(U), 0.4, max_steps=2),
                       "euler_rhs": lambda: (c.euler_rhs(dev(U)), c.sync()),
                       "cfl_dt": lambda: c.cfl_dt(dev(U), 0.4)}.items():
        with pytest.raises(B.T7Error) as ei:
            call()
        assert ei.value.status == want, (name, str(ei.value))
        idx = reported_index(ei.value)
        ry, rx = divmod(idx, nx)
        # within the stencil reach (4 cells per stage) of the poisoned cell
        assert abs(ry - y) <= 24 and abs(rx - x) <= 24, (name, str(ei.value))
        steps, _ = c.run(dev(U0), 0.4, max_steps=2)
        assert steps == 2, name


@pytest.mark.parametrize("prec,dtype", [(B.T7_F64, torch.float64), (B.T7_F32, torch.float32)], ids=["f64", "f32"])
@pytest.mark.parametrize("kind", KINDS)
def test_batch_poisoned_tube_reported(prec, dtype, kind):
    """One poisoned cell in tube 5 of a 12-tube batch: the status names an
    index inside that tube (or its boundary face), and a clean batch run on
    the same context afterwards succeeds."""
    U0, off, dx, _ = I.riemann_tube_batch(3, 12, 40, 120)
    U = U0.copy()
    k = int(off[5] + (off[6] - off[5]) // 3)
    want = poison(U, kind, k)
    c = B.Context(B.T7_EULER1D, U.shape[1], 1.0, prec=prec, bc=(1, 1, 0, 0))
    with pytest.raises(B.T7Error) as ei:
        c.batch_run(torch.tensor(U, dtype=dtype, device="cuda"), off, dx, 0.01, 0.5, max_steps=3)
    assert ei.value.status == want, str(ei.value)
    assert off[5] - 1 <= reported_index(ei.value) <= off[6], str(ei.value)
    steps, t = c.batch_run(torch.tensor(U0, dtype=dtype, device="cuda"), off, dx, 0.01, 0.5, max_steps=3)
    assert np.all(steps == 3)
