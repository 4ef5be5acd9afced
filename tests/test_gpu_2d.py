"""GPU parity of the 2D Euler path (dimension by dimension) against the CPU oracle.

FP64 is bit-identical to the oracle (same operation order, including the
component permutation of the y frame): RHS, masks of both sweeps, RK3 steps and
whole runs.  FP32 is checked against the FP64 oracle with tolerances derived
from FP32 rounding.  At the benchmark size (2048^2) the RHS is sampled against
the oracle evaluated on windows around the samples.
"""
import numpy as np
import pytest

import oracle
import oracle_runs
from paper_1808_00037_gb300 import binding as B
from paper_1808_00037_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ZG = (B.T7_BC_ZERO_GRADIENT,) * 4
PER = (B.T7_BC_PERIODIC,) * 4


def ctx(nx, ny, dx, dy, prec=B.T7_F64, bc=ZG):
    return B.Context(B.T7_EULER2D, nx, dx, ny=ny, dy=dy, prec=prec, bc=bc)


def dev(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def host(t):
    return t.double().cpu().numpy()


def case(name, nx, ny):
    if name == "quadrants":
        U, dx, dy, _ = I.quadrants_2d(4, nx, ny)
        return U, dx, dy, ZG
    if name == "smooth":
        U, dx, dy = I.random_smooth_2d(6, nx, ny)
        return U, dx, dy, PER
    raise ValueError(name)


@pytest.mark.parametrize("name", ["quadrants", "smooth"])
@pytest.mark.parametrize("nx,ny", [(1, 1), (1, 9), (9, 1), (2, 3), (5, 7), (32, 29), (61, 37), (96, 64)])
def test_rhs_2d_f64_bitexact(name, nx, ny):
    U, dx, dy, bc = case(name, nx, ny)
    ro, (ax, ay), (mxo, myo) = oracle.rhs_2d(U, dx, dy, bc=bc, want_masks=True)
    c = ctx(nx, ny, dx, dy, bc=bc)
    rg, (mxg, myg) = c.euler_rhs(dev(U), want_masks=True)
    c.sync()
    assert np.array_equal(mxg.cpu().numpy(), mxo)
    assert np.array_equal(myg.cpu().numpy(), myo)
    assert np.array_equal(host(rg), ro)


@pytest.mark.parametrize("name", ["quadrants", "smooth"])
def test_rk3_step_2d_f64_bitexact(name):
    nx, ny = 70, 45
    U, dx, dy, bc = case(name, nx, ny)
    dt = oracle.cfl_dt_2d(U, dx, dy, 0.4)
    Uo = U.copy()
    st = oracle.lib().or_rk3_step_2d(oracle._ptr(Uo), nx, ny, dx, dy, 1.4, 1e-5, -1.0, -1.0,
                                     oracle._ptr(np.asarray(bc, np.int32)), dt)
    assert st == 0
    c = ctx(nx, ny, dx, dy, bc=bc)
    assert c.cfl_dt(dev(U), 0.4) == dt
    Ug = dev(U)
    c.rk3_step(Ug, dt)
    c.sync()
    assert np.array_equal(host(Ug), Uo)


def test_quadrant_run_2d_f64_bitexact():
    """Four-quadrant Riemann data, transmissive boundaries, CFL 0.4, 40 steps."""
    U, dx, dy, _ = I.quadrants_2d(11, 96, 80)
    Uo, so, to, st = oracle.run_2d(U, dx, dy, cfl=0.4, max_steps=40)
    assert st == 0
    c = ctx(96, 80, dx, dy)
    Ug = dev(U)
    sg, tg = c.run(Ug, 0.4, max_steps=40)
    assert (sg, tg) == (so, to)
    assert np.array_equal(host(Ug), Uo)


@pytest.mark.parametrize("row", oracle_runs.rows("euler2d"), ids=lambda r: r[0])
def test_long_quadrant_runs_f64_bitexact(row):
    """The 2D gate's long runs on the benchmark's quadrant states: 256^2 for
    500 steps and the full 2048^2 for 20 steps, transmissive, CFL 0.4.  The
    FP64 end state, step count and time equal the oracle's bit for bit (the
    oracle's end state is stored as a hash: the runs take minutes on the CPU,
    golden/make_runs.py)."""
    name, seed, nx, ny, steps, t_end, digest = row
    U, dx, dy, _ = I.quadrants_2d(seed, nx, ny)
    c = ctx(nx, ny, dx, dy)
    Ug = dev(U)
    sg, tg = c.run(Ug, 0.4, max_steps=steps)
    assert (sg, tg) == (steps, t_end)
    assert oracle_runs.state_hash(host(Ug)) == digest
    c.close()


def test_smooth_run_2d_f32_tolerance():
    """Smooth periodic 2D flow: FP32 within 1e-5 relative L1 of the FP64 oracle."""
    U, dx, dy = I.random_smooth_2d(3, 64, 64)
    Uo, so, to, st = oracle.run_2d(U, dx, dy, cfl=0.4, t_end=0.05, bc=PER)
    c = ctx(64, 64, dx, dy, prec=B.T7_F32, bc=PER)
    Ug = dev(U, torch.float32)
    sg, tg = c.run(Ug, 0.4, t_end=0.05)
    assert tg == pytest.approx(0.05, abs=1e-12)
    got = host(Ug)
    for k in range(4):
        assert np.abs(got[k] - Uo[k]).sum() / np.abs(Uo[k]).sum() < 1e-5, k


def test_quadrant_run_2d_f32():
    U, dx, dy, _ = I.quadrants_2d(11, 96, 80)
    Uo, so, to, st = oracle.run_2d(U, dx, dy, cfl=0.4, max_steps=40)
    c = ctx(96, 80, dx, dy, prec=B.T7_F32)
    Ug = dev(U, torch.float32)
    c.run(Ug, 0.4, max_steps=40)
    got = host(Ug)
    assert np.abs(got[0] - Uo[0]).sum() / np.abs(Uo[0]).sum() < 1e-3


def test_2d_conservation_periodic_f32_f64():
    U, dx, dy, _ = I.quadrants_2d(5, 128, 96)
    for prec, dtype, tol in ((B.T7_F64, torch.float64, 1e-12), (B.T7_F32, torch.float32, 2e-6)):
        c = ctx(128, 96, dx, dy, prec=prec, bc=PER)
        Ug = dev(U, dtype)
        s0 = Ug.double().sum(dim=(1, 2))
        c.run(Ug, 0.4, max_steps=5)
        s1 = Ug.double().sum(dim=(1, 2))
        assert torch.all(torch.abs(s1 - s0) <= tol * torch.abs(Ug.double()).sum(dim=(1, 2)))


def test_full_size_2d_rhs_sampled_f64():
    """2048^2 four-quadrant data (the benchmark's 2D size): RHS and masks on
    sampled cells equal the oracle on 25 x 25 windows (the RHS at a cell
    depends on cells within 4 of it along its row and column, plus the global
    alphas, which the oracle computes over the full array)."""
    n = 2048
    U, dx, dy, _ = I.quadrants_2d(4, n, n)
    rho = U[0] * (1.0 + 0.05 * np.sin(np.arange(n) * 0.37))[None, :]  # structure inside the quadrants
    U = I.prim_to_cons_2d(rho, U[1] / U[0], U[2] / U[0], (1.4 - 1.0) * (U[3] - 0.5 * (U[1] ** 2 + U[2] ** 2) / U[0]))
    ax, ay = oracle.alpha_2d(U)
    c = ctx(n, n, dx, dy)
    rg, (mxg, myg) = c.euler_rhs(dev(U), want_masks=True)
    c.sync()
    rg = host(rg)
    rng = np.random.default_rng(1)
    pts = [(0, 0), (n - 1, n - 1), (1023, 1024), (1024, 1023), (5, n - 3)] + [
        tuple(p) for p in rng.integers(0, n, (60, 2))]
    W = 12
    for (y, x) in pts:
        y0, y1 = max(0, y - W), min(n, y + W + 1)
        x0, x1 = max(0, x - W), min(n, x + W + 1)
        win = np.ascontiguousarray(U[:, y0:y1, x0:x1])
        ro, _, (mxo, myo) = oracle.rhs_2d(win, dx, dy, bc=ZG, alpha=(ax, ay), want_masks=True)
        assert np.array_equal(rg[:, y, x], ro[:, y - y0, x - x0]), (y, x)
        # x faces x-1/2 and x+1/2 of row y; y faces of column x
        assert np.array_equal(mxg[:, :, y, x:x + 2].cpu().numpy(), mxo[:, :, y - y0, x - x0:x - x0 + 2])
        assert np.array_equal(myg[:, :, x, y:y + 2].cpu().numpy(), myo[:, :, x - x0, y - y0:y - y0 + 2])
