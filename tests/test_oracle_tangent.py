"""Pins of the oracle's tangent-linear mode (rhs_1d_tl, rk3_step_1d_tl,
run_1d_tl): the directional derivative of the scheme with the stencil
selection and the global Lax-Friedrichs alpha frozen, the reference of the
discrete adjoint.

* The value parts equal the primal oracle bit for bit (same operations).
* Euler's theorem: with alpha and the selection frozen, the Euler flux is
  homogeneous of degree 1 in U and the Roe frame of degree 0 (u and H do not
  change when a state is scaled), so the frozen L is homogeneous of degree 1
  and J U = L(U); for linear advection J u = L(u) exactly.
* Fourth-order central differences of the primal oracle, with alpha passed in
  and the selection checked unchanged at every difference point, agree with
  the derivative to their truncation error (RHS and a whole RK3 step).
"""
import numpy as np
import pytest

import oracle
from paper_1808_00037_gb300 import inputs as I


def _cases():
    U, dx, _ = I.random_euler_smooth(2, 300)
    yield "smooth", oracle.SYS_EULER1D, U, dx, (0, 0)
    U, dx, _ = I.riemann_tube(300, *I.SOD)
    yield "sod", oracle.SYS_EULER1D, U, dx, (1, 1)
    U, dx = I.shu_osher(400)
    yield "shu-osher", oracle.SYS_EULER1D, U, dx, (1, 1)
    U, dx, _ = I.burgers_sine(160)
    yield "burgers", oracle.SYS_BURGERS, U, dx, (0, 0)
    U, dx, _ = I.advection_sine(200)
    yield "advection", oracle.SYS_ADVECTION, U, dx, (0, 0)


@pytest.mark.parametrize("case", list(_cases()), ids=lambda c: c[0])
def test_tl_values_equal_primal(case):
    name, sys_, U, dx, bc = case
    L, alpha, masks = oracle.rhs_1d(sys_, U, dx, bc=bc, want_masks=True)
    rng = np.random.default_rng(1)
    Lt, _ = oracle.rhs_1d_tl(sys_, U, rng.normal(size=U.shape), dx, alpha, masks, bc=bc)
    assert np.array_equal(Lt, L)


@pytest.mark.parametrize("case", [c for c in _cases() if c[0] != "burgers"], ids=lambda c: c[0])
def test_tl_homogeneity(case):
    name, sys_, U, dx, bc = case
    L, alpha, masks = oracle.rhs_1d(sys_, U, dx, bc=bc, want_masks=True)
    _, JU = oracle.rhs_1d_tl(sys_, U, U, dx, alpha, masks, bc=bc)
    if sys_ == oracle.SYS_ADVECTION:
        assert np.array_equal(JU, L)
    else:
        assert np.max(np.abs(JU - L)) <= 1e-11 * np.max(np.abs(L)), name


def _fd4(f, U, w, h):
    return (8 * (f(U + h * w) - f(U - h * w)) - (f(U + 2 * h * w) - f(U - 2 * h * w))) / (12 * h)


@pytest.mark.parametrize("case", list(_cases()), ids=lambda c: c[0])
def test_tl_rhs_against_central_differences(case):
    name, sys_, U, dx, bc = case
    L, alpha, m0 = oracle.rhs_1d(sys_, U, dx, bc=bc, want_masks=True)
    rng = np.random.default_rng(3)
    w = rng.normal(size=U.shape) * (np.abs(U) + 0.1)
    _, Jw = oracle.rhs_1d_tl(sys_, U, w, dx, alpha, m0, bc=bc)

    def f(X):
        r, _, ms = oracle.rhs_1d(sys_, X, dx, bc=bc, alpha=alpha, want_masks=True)
        assert np.array_equal(ms, m0)  # the selection is frozen at +-h, +-2h
        return r
    fd = _fd4(f, U, w, 1e-5)
    assert np.max(np.abs(fd - Jw)) <= 1e-8 * np.max(np.abs(Jw)), name


def test_tl_rk3_step_against_central_differences():
    """A whole step: stages with the primal stage states' alphas and
    selections frozen (the differences reuse them), Shu-Osher form."""
    U, dx, _ = I.random_euler_smooth(4, 256)
    sys_, bc = oracle.SYS_EULER1D, (0, 0)
    dt = 0.5 * dx / oracle.alpha_1d(sys_, U)
    rng = np.random.default_rng(5)
    w = rng.normal(size=U.shape) * np.abs(U)
    U1, dU1 = oracle.rk3_step_1d_tl(sys_, U, w, dx, dt, bc=bc)
    assert np.array_equal(U1, oracle.rk3_step_1d(sys_, U, dx, dt, bc=bc))
    frozen = []
    X = U
    for s in range(3):  # the primal stage states' alphas and masks
        r, a, ms = oracle.rhs_1d(sys_, X, dx, bc=bc, want_masks=True)
        frozen.append((a, ms))
        X = [U + dt * r, 0.75 * U + 0.25 * (X + dt * r), None][s]

    def step(V):
        X = V
        for s, (a, ms) in enumerate(frozen):
            r, _, m2 = oracle.rhs_1d(sys_, X, dx, bc=bc, alpha=a, want_masks=True)
            assert np.array_equal(m2, ms)
            X = [V + dt * r, 0.75 * V + 0.25 * (X + dt * r), (1.0 / 3.0) * V + (2.0 / 3.0) * (X + dt * r)][s]
        return X
    fd = _fd4(step, U, w, 1e-5)
    assert np.max(np.abs(fd - dU1)) <= 1e-8 * np.max(np.abs(dU1))


def test_tl_run_is_repeated_steps():
    U, dx, _ = I.random_euler_smooth(4, 128)
    w = np.random.default_rng(7).normal(size=U.shape)
    dt = 0.4 * dx / oracle.alpha_1d(oracle.SYS_EULER1D, U)
    Ur, dUr = oracle.run_1d_tl(oracle.SYS_EULER1D, U, w, dx, dt, 3, bc=(0, 0))
    X, dX = U, w
    for _ in range(3):
        X, dX = oracle.rk3_step_1d_tl(oracle.SYS_EULER1D, X, dX, dx, dt, bc=(0, 0))
    assert np.array_equal(Ur, X) and np.array_equal(dUr, dX)
