"""Pins of the approximate-dispersion-relation analysis (Sec. "Approximate
dispersion relation analysis") on the oracle: modes u_j = cos(phi j) on a
periodic grid of N = 256 points, Phi = i dx L^_n / (a u^_n).

* With the cutoff disabled (C_T = 1e-300, every stencil kept) TENO7-ext and
  TENO5 are their background linear schemes, whose modified wavenumbers have
  the closed form -i (1 - e^{-i phi}) sum_t c_t e^{i phi (t + o)} (Table co2
  row 0, Table co1 row 0): equal to 1e-12 on every mode, Nyquist included.
* With C_T = 1e-5 both nonlinear schemes follow their linear schemes up to a
  wavenumber and leave them at the same wavenumber, since TENO7-ext uses
  TENO5's smoothness measurement (the paper's reading of its ADR figure).
* Above it TENO7-ext stays closer to the exact Phi = phi than TENO5: its
  resolving wavenumber at 1% and 10% error is higher (the paper's claim of
  lower dissipation and dispersion at high wavenumbers)."""
import numpy as np
import pytest

import oracle

N = 256


def oracle_adr(scheme, CT):
    dx = 1.0 / N
    j = np.arange(N)
    out = []
    with oracle.scheme(scheme):
        for n in range(1, N // 2 + 1):
            u = np.cos(2 * np.pi * n * j / N)
            L, _, _ = oracle.rhs_1d(oracle.SYS_ADVECTION, u[None, :], dx, CT=CT)
            out.append(1j * dx * np.fft.fft(L[0])[n] / np.fft.fft(u)[n])
    return 2 * np.pi * np.arange(1, N // 2 + 1) / N, np.array(out)


def linear_phi(phi, coef, offset):
    return -1j * (1 - np.exp(-1j * phi)) * sum(c * np.exp(1j * phi * (t + offset)) for t, c in enumerate(coef))


def first_departure(a, b, tol=1e-6):
    return int(np.argmax(np.abs(a - b) > tol))


@pytest.fixture(scope="module")
def curves():
    out = {}
    for name, sch in (("t7", oracle.SCHEME_TENO7EXT), ("t5", oracle.SCHEME_TENO5)):
        out[name] = oracle_adr(sch, 1e-5)
        out[name + "lin"] = oracle_adr(sch, 1e-300)
    return out


def test_linear_limits_match_closed_forms(curves):
    phi, l7 = curves["t7lin"]
    _, l5 = curves["t5lin"]
    c7 = oracle.coeffs()[0]
    c5 = oracle.coeffs5()[0]
    assert np.max(np.abs(l7 - linear_phi(phi, c7, -3))) < 1e-12
    assert np.max(np.abs(l5 - linear_phi(phi, c5, -2))) < 1e-12
    # the seventh-order scheme: |Phi - phi| = O(phi^8) at small phi
    assert abs(l7[4] - phi[4]) < 1e-8 and abs(l5[4] - phi[4]) > 10 * abs(l7[4] - phi[4])


def test_nonlinear_schemes_leave_their_linear_schemes_at_the_same_wavenumber(curves):
    phi, a7 = curves["t7"]
    _, a5 = curves["t5"]
    k7 = first_departure(a7, curves["t7lin"][1])
    k5 = first_departure(a5, curves["t5lin"][1])
    assert k7 == k5 and 0.4 * np.pi < phi[k7] < 0.75 * np.pi, (phi[k7], phi[k5])
    assert np.max(np.abs(a7[:k7] - curves["t7lin"][1][:k7])) < 1e-12


def test_teno7ext_resolves_higher_wavenumbers_than_teno5(curves):
    phi, a7 = curves["t7"]
    _, a5 = curves["t5"]
    for tol in (1e-2, 1e-1):
        r7 = phi[np.argmax(np.abs(a7 - phi) > tol)]
        r5 = phi[np.argmax(np.abs(a5 - phi) > tol)]
        assert r7 > r5 + 0.1, (tol, r7, r5)
    # dissipation: Im Phi <= 0 (no anti-dissipation) for both schemes
    assert np.all(a7.imag < 1e-12) and np.all(a5.imag < 1e-12)
