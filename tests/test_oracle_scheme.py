"""Pins of the oracle's scheme against what the paper and the mathematics fix
(scalar problems): recovery of the linear seventh-order upwind scheme on smooth
data, the measured order of accuracy, the exact shift of linear advection,
conservation, mirror symmetry of the '-' split, and non-oscillatory selection
at a jump."""

import numpy as np
import pytest

from paper_1808_00037_gb300 import inputs as I
from test_oracle_tables import reconstruction_coeffs

SEVEN = np.array([float(reconstruction_coeffs(-3, 3)[l]) for l in range(-3, 4)])


def linear_rhs(u, dx):
    """The linear seventh-order upwind scheme for u_t + u_x = 0 on a periodic
    grid, with coefficients from the exact rational derivation."""
    n = u.size
    fh = np.zeros(n)  # face i+1/2
    for t, l in enumerate(range(-3, 4)):
        fh += SEVEN[t] * np.roll(u, -l)
    return -(fh - np.roll(fh, 1)) / dx


@pytest.mark.parametrize("n", [80, 160, 320])
def test_linear_scheme_recovered_on_smooth_data(orc, n):
    U, dx, x = I.advection_sine(n)
    r, alpha, masks = orc.rhs_1d(orc.SYS_ADVECTION, U, dx, want_masks=True)
    assert alpha == 1.0
    assert np.all(masks == 0b11111)  # every face picks f0 (all stencils smooth)
    ref = linear_rhs(U[0], dx)
    assert np.max(np.abs(r[0] - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_spatial_order_is_seven(orc):
    errs = []
    ns = [20, 40, 80, 160]
    for n in ns:
        U, dx, x = I.advection_sine(n)
        r, _, _ = orc.rhs_1d(orc.SYS_ADVECTION, U, dx)
        errs.append(np.max(np.abs(r[0] + np.pi * np.cos(np.pi * x))))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 6.8), orders


def test_full_run_order_with_refined_dt(orc):
    """Gaussian-free variant of the smooth advection test: sin(pi x) advected one
    period with dt ~ dx^(7/3) so the RK3 error stays below the spatial error."""
    errs = []
    for n in [20, 40, 80]:
        U, dx, x = I.advection_sine(n)
        dt = 0.2 * dx * (dx / 0.1) ** (4.0 / 3.0)
        Uf, steps, t, st = orc.run_1d(orc.SYS_ADVECTION, U, dx, t_end=2.0, dt_fixed=dt)
        assert t == pytest.approx(2.0, abs=1e-12)
        errs.append(np.max(np.abs(Uf[0] - np.sin(np.pi * x))))  # exact shift: back to u0 at t = 2
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 6.5), orders


def test_advection_config_exact_shift(orc):
    U, dx, x = I.advection_sine(200)
    Uf, steps, t, st = orc.run_1d(orc.SYS_ADVECTION, U, dx, t_end=2.0, cfl=0.2)
    assert steps in (1000, 1001) and t == pytest.approx(2.0, abs=1e-12)
    # the error is the RK3 time error (~ t dt^3 pi^4 / 24); spatial error is ~1e-13
    assert np.max(np.abs(Uf[0] - np.sin(np.pi * x))) < 2e-7


def test_gaussian_and_sin3_recover_linear_scheme(orc):
    for gen in (I.advection_gaussian, I.advection_sin3):
        U, dx, x = gen(320)
        r, _, masks = orc.rhs_1d(orc.SYS_ADVECTION, U, dx, want_masks=True)
        ref = linear_rhs(U[0], dx)
        frac = np.mean(masks[0] == 0b11111)
        # with eps = dx^3 the smooth fields (critical points included) keep f0
        assert frac == 1.0, (gen.__name__, frac)
        assert np.max(np.abs(r[0] - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_reconstruct_mirror_is_reversal(orc):
    rng = np.random.default_rng(5)
    n = 64
    v = np.cumsum(rng.normal(size=n + 8))
    v[30:] += 5.0  # a jump
    fp, d3p, D5p = orc.teno7_reconstruct(v[::-1].copy(), +1, eps=1e-6)
    fm, d3m, D5m = orc.teno7_reconstruct(v, -1, eps=1e-6)
    # '-' at face f of v is '+' at face n - f of the reversed sequence
    assert np.array_equal(fm, fp[::-1])
    assert np.array_equal(D5m, D5p[::-1])
    assert np.array_equal(d3m, d3p[::-1])


def test_reconstruct_jump_never_crosses(orc):
    """A clean jump: every face value is one of the two plateau values (no
    stencil crosses the discontinuity), and the face at the jump takes the
    upwind (left) value."""
    n = 40
    v = np.where(np.arange(-4, n + 4) < 20, 0.0, 1.0)
    fh, d3, D5 = orc.teno7_reconstruct(v, +1, eps=(1.0 / n) ** 3)
    faces = np.arange(-1, n)  # face i+1/2
    near = np.minimum(np.abs(fh), np.abs(fh - 1.0))
    assert np.max(near) < 1e-14
    assert abs(fh[faces == 19][0]) < 1e-14  # face 19+1/2: upwind cell 19 is on the left plateau


def test_reconstruct_polynomial_exact(orc):
    """Point values that are cell averages of a degree-6 polynomial are
    reconstructed exactly at the faces by f0 (the seventh-order polynomial)."""
    n = 50
    dx = 1.0 / n
    c = [1.0, 2.0, -0.5, 0.3, 0.2, -0.1, 0.05]
    P = np.polynomial.Polynomial(c)
    Pi = P.integ()
    xl = (np.arange(-4, n + 4)) * dx
    v = (Pi(xl + dx) - Pi(xl)) / dx  # cell averages over [x_l, x_l + dx]
    fh, d3, D5 = orc.teno7_reconstruct(v, +1, eps=dx**3)
    assert np.all(D5 == 0b11111)
    xf = (np.arange(-1, n) + 1) * dx  # face i+1/2 at x = (i+1) dx
    assert np.max(np.abs(fh - P(xf))) < 1e-12


def test_uniform_state_is_steady(orc):
    n = 37
    for sys, U in ((orc.SYS_ADVECTION, np.full((1, n), 0.7)),
                   (orc.SYS_BURGERS, np.full((1, n), -0.3)),
                   (orc.SYS_EULER1D, I.prim_to_cons_1d(np.full(n, 0.9), np.full(n, 0.4), np.full(n, 2.0)))):
        for bc in ((0, 0), (1, 1)):
            r, _, _ = orc.rhs_1d(sys, U, 0.1, bc=bc)
            assert np.all(r == 0.0)


def test_periodic_conservation(orc):
    rng = np.random.default_rng(11)
    n = 200
    u = np.sin(2 * np.pi * np.arange(n) / n) + (np.arange(n) > n // 2) + 0.1 * rng.normal(size=n)
    for sys, a in ((orc.SYS_ADVECTION, 1.0), (orc.SYS_ADVECTION, -0.7), (orc.SYS_BURGERS, 1.0)):
        r, _, _ = orc.rhs_1d(sys, u[None, :], 0.01, a=a)
        assert abs(r.sum()) <= 1e-13 * np.abs(r).sum()


def test_advection_reflection(orc):
    """u_t + a u_x = 0 reflected in x is u_t - a u_x = 0: the '-' split of the
    reflected problem must mirror the '+' split of the original."""
    rng = np.random.default_rng(3)
    n = 96
    u = np.cumsum(rng.normal(size=n)) * 0.1
    u[40:55] += 1.0
    r1, _, m1 = orc.rhs_1d(orc.SYS_ADVECTION, u[None, :], 0.05, a=1.3, want_masks=True)
    r2, _, m2 = orc.rhs_1d(orc.SYS_ADVECTION, u[::-1][None, :].copy(), 0.05, a=-1.3, want_masks=True)
    assert np.allclose(r2[0][::-1], r1[0], rtol=0, atol=1e-12 * np.abs(r1).max())
    # face f of the original <-> face n - f of the reflection, '+' <-> '-'
    assert np.array_equal(m2[1, 0][::-1], m1[0, 0])
    assert np.array_equal(m2[0, 0][::-1], m1[1, 0])


def test_burgers_smooth_order(orc):
    """Inviscid Burgers, u0 = 1/2 + sin(pi x) on [0, 2): before the shock time the
    RHS error against -u u_x of the exact field has order ~7."""
    errs = []
    for n in [40, 80, 160]:
        U, dx, x = I.burgers_sine(n)
        r, alpha, _ = orc.rhs_1d(orc.SYS_BURGERS, U, dx)
        assert alpha == np.max(np.abs(U[0]))  # global Lax-Friedrichs alpha = max |f'(u)|
        u = U[0]
        errs.append(np.max(np.abs(r[0] + u * np.pi * np.cos(np.pi * x))))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 6.0), orders
