"""Pins of the oracle on the paper's remaining scalar and Euler cases: the
sin^3 field with second-order critical points (Eq. init_LinAdv2), the
four-wave field (Eq. init_LinAdv3, N = 400, t = 2), the inviscid Burgers
equation before and after the shock forms (N = 160, t = 0.5/pi and 1.5/pi)
and the Titarev-Toro shock / high-frequency entropy-wave case (Eq. c_se,
N = 400, t = 5).  The paper prints only plots for these; the pins are closed
forms (exact derivatives, the exact Burgers solution by characteristics, the
Rankine-Hugoniot shock speed), invariants (bounds, total variation,
conservation) and the TENO5 comparison the paper draws."""
import numpy as np
import pytest

import oracle
from paper_1808_00037_gb300 import inputs as I


def tv(u):
    return float(np.abs(np.diff(np.concatenate([u, u[:1]]))).sum())


def test_sin3_critical_points_keep_seventh_order():
    """u = sin(pi x)^3 has points with u' = u'' = 0, u''' != 0.  The cutoff
    keeps every stencil (all faces select the seventh-order polynomial) from
    N = 20 on, and the RHS error against the exact -u_x has order 7."""
    errs = []
    for n in (20, 40, 80, 160, 320):
        U, dx, x = I.advection_sin3(n)
        r, _, m = oracle.rhs_1d(oracle.SYS_ADVECTION, U, dx, want_masks=True)
        assert np.all(m[0] == 31)
        exact = -3.0 * np.pi * np.sin(np.pi * x) ** 2 * np.cos(np.pi * x)
        errs.append(np.max(np.abs(r[0] - exact)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders[1:] > 6.9) and np.all(orders < 7.2), orders


def test_four_wave_bounded_and_sharper_than_teno5():
    """N = 400, CFL 0.2, one period (t = 2): the solution stays inside the
    initial range to 1e-3, its total variation does not grow, and its L1
    error is below TENO5's on the same run."""
    U, dx, x = I.four_wave(400)
    assert U.min() == 0.0 and U.max() == 1.0
    Uf, steps, t, st = oracle.run_1d(oracle.SYS_ADVECTION, U, dx, t_end=2.0, cfl=0.2)
    assert st == 0 and t == 2.0
    assert Uf.min() > -1e-3 and Uf.max() < 1.0 + 1e-3
    assert tv(Uf[0]) <= tv(U[0])
    with oracle.scheme(oracle.SCHEME_TENO5):
        U5, _, _, _ = oracle.run_1d(oracle.SYS_ADVECTION, U, dx, t_end=2.0, cfl=0.2)
    assert np.mean(np.abs(Uf - U)) < np.mean(np.abs(U5 - U))


def burgers_exact(x, t):
    """u(x, t) of u_t + (u^2/2)_x = 0, u0 = 1/2 + sin(pi x), before the shock
    time 1/pi: the root of u = 1/2 + sin(pi (x - u t)) by Newton's method."""
    u = 0.5 + np.sin(np.pi * x)
    for _ in range(60):
        s = np.pi * (x - u * t)
        u = u - (u - 0.5 - np.sin(s)) / (1.0 + np.pi * t * np.cos(s))
    return u


def test_burgers_smooth_run_against_characteristics():
    """t = 0.5/pi with dt refined as dx^(7/3): the error against the exact
    solution falls at order ~7."""
    T = 0.5 / np.pi
    errs = []
    for n in (80, 160, 320):
        U, dx, x = I.burgers_sine(n)
        cfl = 0.5 * (dx / (2.0 / 40)) ** (4.0 / 3.0)
        Uf, _, t, st = oracle.run_1d(oracle.SYS_BURGERS, U, dx, t_end=T, cfl=cfl)
        assert st == 0 and t == pytest.approx(T, abs=1e-15)
        errs.append(np.max(np.abs(Uf[0] - burgers_exact(x, T))))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 6.5), orders


def test_burgers_shocked_run_bounded_and_conservative():
    """t = 1.5/pi (after the shock forms), N = 160, CFL 0.5: values stay in
    the initial range [-1/2, 3/2] to 1e-3, total variation does not grow and
    the periodic sum is conserved to round-off."""
    U, dx, x = I.burgers_sine(160)
    Uf, _, t, st = oracle.run_1d(oracle.SYS_BURGERS, U, dx, t_end=1.5 / np.pi, cfl=0.5)
    assert st == 0
    assert Uf.min() > -0.5 - 1e-3 and Uf.max() < 1.5 + 1e-3
    assert tv(Uf[0]) <= tv(U[0])
    assert abs(Uf.sum() - U.sum()) <= 1e-12 * np.abs(U).sum()
    # the shock has formed: the largest jump between neighbours is O(1)
    assert np.max(np.abs(np.diff(Uf[0]))) > 0.5


def test_titarev_toro_shock_position():
    """N = 400 on [0, 10], t = 5: the run stays physical, and the shock (the
    rightmost cell with p above the midpoint of 1 and 1.805) sits within 0.1
    of 0.5 + 5 S, S the Rankine-Hugoniot speed of the printed post-shock state
    into (1, 0, 1) -- the left state is exactly that shock's downstream state."""
    U, dx, x = I.titarev_toro(400)
    gamma = 1.4
    p2 = 1.805
    Ms = np.sqrt(1.0 + (gamma + 1.0) / (2.0 * gamma) * (p2 - 1.0))
    S = Ms * np.sqrt(gamma)
    rho2 = (gamma + 1.0) * Ms**2 / ((gamma - 1.0) * Ms**2 + 2.0)
    u2 = S * (1.0 - 1.0 / rho2)
    assert rho2 == pytest.approx(1.515695, abs=2e-5) and u2 == pytest.approx(0.523346, abs=5e-5)
    Uf, steps, t, st = oracle.run_1d(oracle.SYS_EULER1D, U, dx, t_end=5.0, cfl=0.5, bc=(1, 1))
    assert st == 0 and t == 5.0
    rho, u, p = I.cons_to_prim_1d(Uf)
    assert rho.min() > 0.9 and p.min() > 0.9
    xs = x[np.nonzero(p > 0.5 * (1.0 + p2))[0].max()]
    assert abs(xs - (0.5 + 5.0 * S)) < 0.1, (xs, 0.5 + 5.0 * S)
