"""Pins of the oracle's TENO5 baseline (the fifth-order TENO scheme the paper
compares with): Table co1 as printed (exact rationals, nearest doubles), the
selection by a face's own cutoff bits, recovery of the fifth-order linear
upwind scheme on smooth data with measured order ~5, non-crossing of a jump,
and the Sod tube against the exact solution."""
from fractions import Fraction as Fr
from pathlib import Path

import numpy as np

import oracle
from oracle import riemann
from paper_1808_00037_gb300 import inputs as I
from test_oracle_tables import reconstruction_coeffs

GOLD = Path(__file__).parent / "golden"
FIVE = np.array([float(reconstruction_coeffs(-2, 2)[l]) for l in range(-2, 3)])


def test_co1_coefficients_and_selection():
    rows = [l.split() for l in (GOLD / "table_co1.txt").read_text().splitlines() if l and not l.startswith("#")]
    C = oracle.coeffs5()
    for key, *coef in rows:
        bits = int(key[0]) | (int(key[1]) << 1) | (int(key[2]) << 2)
        r = oracle.select5(bits)
        assert [C[r, t] for t in range(5)] == [float(Fr(x)) for x in coef], key
    assert oracle.select5(0) == -1


def test_teno5_recovers_fifth_order_linear_scheme():
    errs = []
    with oracle.scheme(oracle.SCHEME_TENO5):
        for n in (40, 80, 160, 320):
            U, dx, x = I.advection_sine(n)
            r, _, m = oracle.rhs_1d(oracle.SYS_ADVECTION, U, dx, want_masks=True)
            assert np.all(m == 0b111)
            fh = sum(FIVE[t] * np.roll(U[0], -(t - 2)) for t in range(5))
            ref = -(fh - np.roll(fh, 1)) / dx
            assert np.max(np.abs(r[0] - ref)) <= 1e-12 * np.max(np.abs(ref))
            errs.append(np.max(np.abs(r[0] + np.pi * np.cos(np.pi * x))))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 4.8) and np.all(orders < 5.3), orders


def test_teno5_jump_never_crosses():
    n = 40
    v = np.where(np.arange(-4, n + 4) < 20, 0.0, 1.0)
    with oracle.scheme(oracle.SCHEME_TENO5):
        fh, d3, D5 = oracle.teno7_reconstruct(v, +1, eps=1e-40)
    assert np.max(np.minimum(np.abs(fh), np.abs(fh - 1.0))) < 1e-14


def test_teno5_sod_against_exact():
    U, dx, x = I.riemann_tube(200, *I.SOD)
    with oracle.scheme(oracle.SCHEME_TENO5):
        Uf, steps, t, st = oracle.run_1d(oracle.SYS_EULER1D, U, dx, t_end=0.2, cfl=0.6, bc=(1, 1))
    rho, _, _ = riemann.sample(*I.SOD, (x - 0.5) / 0.2)
    err5 = np.mean(np.abs(Uf[0] - rho))
    assert err5 < 6e-3
    Uf7, _, _, _ = oracle.run_1d(oracle.SYS_EULER1D, U, dx, t_end=0.2, cfl=0.6, bc=(1, 1))
    assert oracle.lib().or_get_scheme() == oracle.SCHEME_TENO7EXT
    assert not np.array_equal(Uf, Uf7)


def flat_faces(U, bc):
    """Faces j+1/2, j = -1 .. n-1, whose cells j-2 .. j+3 hold one constant
    state (ghost cells by the boundary condition)."""
    P = np.pad(U, ((0, 0), (4, 4)), mode="wrap" if bc[0] == 0 else "edge")
    n = U.shape[1]
    flat = np.ones(n + 1, bool)
    for d in range(-2, 4):  # cell j + d for j = -1 .. n-1 sits at padded index j + d + 4
        flat &= np.all(P[:, 3 + d:3 + d + n + 1] == P[:, 3:3 + n + 1], axis=0)
    return flat


def test_teno5_decides_on_roundoff_in_constant_states():
    """On Sod's constant right state TENO5 (epsilon 1e-40) cuts a stencil of
    one characteristic field: beta_2 is the square of the rounding error of
    3 w, and against 1e-40 that decides the cutoff.  TENO7-ext's epsilon =
    dx^3 keeps every stencil on faces whose neighbours are flat too (the
    motivation for redefining epsilon, Sec. "The parameter epsilon")."""
    U, dx = I.riemann_tube(1600, *I.SOD)[:2]
    flat = flat_faces(U, (1, 1))
    with oracle.scheme(oracle.SCHEME_TENO5):
        _, _, m5 = oracle.rhs_1d(oracle.SYS_EULER1D, U, dx, bc=(1, 1), want_masks=True)
    assert np.any(m5[:, :, flat] != 7)
    _, _, m7 = oracle.rhs_1d(oracle.SYS_EULER1D, U, dx, bc=(1, 1), want_masks=True)
    inner = np.zeros_like(flat)
    inner[1:-1] = flat[1:-1] & flat[:-2] & flat[2:]
    assert inner.sum() > 1500
    assert np.all(m7[:, :, inner] == 31)
