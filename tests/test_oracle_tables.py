"""Pins of the oracle's constant tables against the paper and the mathematics.

* Table co2 rows are re-derived with exact rational arithmetic: each row must be
  THE unique reconstruction of the point value h(x_{i+1/2}) from the point
  values f_l, where f is the cell average of h (Eq. flux), on the contiguous
  stencil spanned by the row's non-zero entries.  The oracle's doubles must be
  the nearest doubles to those rationals, and the golden copy of the printed
  table must equal them.
* Table co1 and Eq. 3_rd are checked for mutual consistency (the fifth-order
  TENO weights of Eq. TENO_W turn the three candidate fluxes into Table co1).
* Table co3 is enumerated over all 32 binary vectors, against the golden copy of
  the printed patterns and against the rule the paper states for it: never use
  a stencil judged non-smooth, prefer interpolation over extrapolation, then the
  widest stencil.
"""
from fractions import Fraction as Fr
from pathlib import Path

import numpy as np

GOLD = Path(__file__).parent / "golden"


def _rows(name):
    out = []
    for line in (GOLD / name).read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            out.append(line.split())
    return out


def reconstruction_coeffs(lo, hi):
    """Exact c_l (l = lo..hi, offsets from i) with sum_l c_l avg_l(h) = h(1/2)
    for every polynomial h of degree <= hi-lo (cell width 1, x_i = 0)."""
    K = hi - lo + 1
    cells = list(range(lo, hi + 1))
    A = [[(Fr(2 * l + 1, 2) ** (p + 1) - Fr(2 * l - 1, 2) ** (p + 1)) / (p + 1) for l in cells] for p in range(K)]
    b = [Fr(1, 2) ** p for p in range(K)]
    # Gauss-Jordan in exact arithmetic
    M = [row[:] + [bb] for row, bb in zip(A, b)]
    for col in range(K):
        piv = next(r for r in range(col, K) if M[r][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        pv = M[col][col]
        M[col] = [x / pv for x in M[col]]
        for r in range(K):
            if r != col and M[r][col] != 0:
                f = M[r][col]
                M[r] = [x - f * y for x, y in zip(M[r], M[col])]
    return {l: M[k][K] for k, l in enumerate(cells)}


GOLD_CO2 = [[Fr(x) for x in r] for r in _rows("table_co2.txt")]


def support(row):
    nz = [t - 3 for t, c in enumerate(row) if c != 0]
    return min(nz), max(nz)


def test_golden_co2_rows_are_exact_reconstructions():
    orders = []
    for m, row in enumerate(GOLD_CO2):
        lo, hi = support(row)
        exact = reconstruction_coeffs(lo, hi)
        for t in range(7):
            l = t - 3
            assert row[t] == exact.get(l, Fr(0)), (m, l)
        orders.append(hi - lo + 1)
    # orders printed under Table co2: 7; 6, 6; 5, 5, 5; 4 x 4; 3 x 3
    assert orders == [7, 6, 6, 5, 5, 5, 4, 4, 4, 4, 3, 3, 3]


def test_oracle_coefficients_are_nearest_doubles(orc):
    C = orc.coeffs()
    for m, row in enumerate(GOLD_CO2):
        for t in range(7):
            assert C[m, t] == float(row[t]), (m, t)


def test_candidate_fluxes_and_table_co1_consistent():
    rows = {r[0]: [Fr(x) for x in r[1:]] for r in _rows("candidate_fluxes.txt")}
    S = [rows["S0"], rows["S1"], rows["S2"]]
    d = rows["d"]
    for k, (lo, hi) in enumerate([(-2, 0), (-1, 1), (0, 2)]):
        ex = reconstruction_coeffs(lo, hi)
        assert [ex.get(l, Fr(0)) for l in range(-2, 3)] == S[k]
    for r in _rows("table_co1.txt"):
        bits = [int(c) for c in r[0]]
        expect = [Fr(x) for x in r[1:]]
        den = sum(dk * bk for dk, bk in zip(d, bits))
        comb = [sum(d[k] * bits[k] * S[k][t] for k in range(3)) / den for t in range(5)]
        assert comb == expect, r[0]
    # all three smooth: the fifth-order upwind scheme on i-2..i+2
    ex5 = reconstruction_coeffs(-2, 2)
    assert [ex5[l] for l in range(-2, 3)] == [Fr(x) for x in _rows("table_co1.txt")[0][1:]]


def _golden_co3():
    pats = []
    for pat, m in _rows("table_co3.txt"):
        pats.append((pat, None if m == "none" else int(m)))
    return pats


def _vec(D):
    return [(D >> (4 - c)) & 1 for c in range(5)]


def rule_select(vec):
    """The selection rule stated with Table co3, from the stencil supports only:
    a candidate is admissible iff every three-point stencil inside its support is
    smooth; prefer admissible candidates whose support holds both i and i+1
    (interpolation), then the widest one."""
    if vec[1] == vec[2] == vec[3] == 0:
        return None
    adm = []
    for m, row in enumerate(GOLD_CO2):
        lo, hi = support(row)
        windows = [l for l in range(lo, hi - 1)]  # stencils [l, l+2]
        if all(vec[l + 3] == 1 for l in windows):
            adm.append((m, lo, hi))
    interp = [c for c in adm if c[1] <= 0 and c[2] >= 1]
    pool = interp if interp else adm
    width = max(c[2] - c[1] for c in pool)
    best = [c[0] for c in pool if c[2] - c[1] == width]
    assert len(best) == 1, (vec, best)
    return best[0]


def test_table_co3_exhaustive(orc):
    pats = _golden_co3()
    for D in range(32):
        vec = _vec(D)
        matches = [m for pat, m in pats if all(p == "*" or int(p) == b for p, b in zip(pat, vec))]
        assert len(matches) == 1, (vec, matches)  # no gaps, no overlaps
        expect = matches[0]
        got = orc.select(D)
        assert (got if got >= 0 else None) == expect, vec
        assert rule_select(vec) == expect, vec


def test_tie_rules(orc):
    # (1,1,0,1,1) -> f6 (interpolation) rather than f9; (1,1,0,1,0) -> f10 rather than f9
    assert orc.select(0b11011) == 6
    assert orc.select(0b11010) == 10
    # central triple never all zero for finite data: sum chi = 1 => max chi >= 1/3 > CT
    for D in (0b00000, 0b00001, 0b10000, 0b10001):
        assert orc.select(D) == -1


def test_face_bits_hand_computed(orc):
    eps = 1e-6
    bits, beta = orc.face_bits([2.0] * 5, eps)
    assert bits == 0b111 and np.all(beta == 0.0)
    # linear data: all three betas equal (= 1), tau = 0 -> all smooth
    bits, beta = orc.face_bits([0.0, 1.0, 2.0, 3.0, 4.0], eps)
    assert bits == 0b111 and np.allclose(beta, [1.0, 1.0, 1.0], rtol=0, atol=1e-15)
    # jump between f_i and f_{i+1}: only S0 = {i-2, i-1, i} is smooth
    bits, beta = orc.face_bits([0.0, 0.0, 0.0, 1.0, 1.0], eps)
    assert bits == 0b001
    assert beta[0] == 0.0 and abs(beta[1] - 4.0 / 3.0) < 1e-15 and abs(beta[2] - 10.0 / 3.0) < 1e-15
    # jump between f_{i-1} and f_i: only S2 = {i, i+1, i+2} is smooth
    bits, beta = orc.face_bits([1.0, 1.0, 0.0, 0.0, 0.0], eps)
    assert bits == 0b100
    assert abs(beta[0] - 10.0 / 3.0) < 1e-15 and abs(beta[1] - 4.0 / 3.0) < 1e-15 and beta[2] == 0.0
    # jump between f_{i-2} and f_{i-1}: S1 and S2 smooth, S0 cut
    bits, _ = orc.face_bits([1.0, 0.0, 0.0, 0.0, 0.0], eps)
    assert bits == 0b110


def test_cutoff_threshold_direction(orc):
    """delta_k = 0 exactly when chi_k < CT (Eq. seclect): sweep CT across the
    chi of a fixed window and watch the bit switch at chi."""
    w = [0.0, 0.1, 0.25, 0.9, 1.0]
    eps = 1e-6
    bits_lo, beta = orc.face_bits(w, eps, CT=1e-30)
    assert bits_lo == 0b111
    tau = abs(beta[0] - beta[2])
    gam = (1.0 + tau / (beta + eps)) ** 6
    chi = gam / gam.sum()
    k = int(np.argmin(chi))
    below, _ = orc.face_bits(w, eps, CT=chi[k] * (1 + 1e-9))
    above, _ = orc.face_bits(w, eps, CT=chi[k] * (1 - 1e-9))
    assert (below >> k) & 1 == 0 and (above >> k) & 1 == 1


# Marginal cutoff windows, evaluated by hand in exact arithmetic.  The window
# w = (f_{i-2}, .., f_{i+2}) = (0, 0, 1, 2, 0) gives, by Eq. smooth_expl,
#   beta_0 = 1/4 (0 - 0 + 3)^2 + 13/12 (0 - 0 + 1)^2   = 9/4 + 13/12   = 10/3
#   beta_1 = 1/4 (0 - 2)^2     + 13/12 (0 - 2 + 2)^2   = 1 + 0         = 1
#   beta_2 = 1/4 (3 - 8 + 0)^2 + 13/12 (1 - 4 + 0)^2   = 25/4 + 39/4   = 16
# and tau_5 = |beta_0 - beta_2| = 38/3 (Eq. tau5).  With C = 1, q = 6
# (Eq. TENO1), gamma_k = g_k^6 where g_k = 1 + tau_5 / (beta_k + eps):
#   eps = 1/6:  g = (1 + 76/21, 1 + 76/7, 1 + 76/97) = (97/21, 83/7, 173/97)
#               chi_2 = g_2^6 / sum g^6 = 1.1541e-5, between C_T and 2 C_T
#   eps = 1/8:  g = (1 + 304/83, 1 + 304/27, 1 + 304/387) = (387/83, 331/27, 691/387)
#               chi_2 = 9.517e-6, just below C_T
# (Eq. norm), so by Eq. seclect with C_T = 1e-5 the first keeps all three
# stencils (bits 111) and the second cuts stencil 2 (bits 011).  chi_0 and
# chi_1 are 3.5e-3 / 3.0e-3 and 0.9965 / 0.9970, far from the threshold.
# Each of these mistakes changes the bits of one of the two windows:
# q = 2, 4 or 8; C = 0; no normalisation (delta from gamma itself); tau from
# |beta_0 - beta_1| or |beta_1 - beta_2|; the window read in reverse order.
MARGINAL_W = [0.0, 0.0, 1.0, 2.0, 0.0]
MARGINAL_BETA = (Fr(10, 3), Fr(1), Fr(16))
MARGINAL_CASES = [
    # eps, (g_0, g_1, g_2), chi_2 bounds, bits
    (Fr(1, 6), (Fr(97, 21), Fr(83, 7), Fr(173, 97)), (Fr(115, 10**7), Fr(116, 10**7)), 0b111),
    (Fr(1, 8), (Fr(387, 83), Fr(331, 27), Fr(691, 387)), (Fr(95, 10**7), Fr(96, 10**7)), 0b011),
]


def test_cutoff_marginal_windows_exact(orc):
    """Eqs. smooth_expl, tau5, TENO1 (C = 1, q = 6), norm and seclect pinned
    by two windows whose smallest chi lies within a factor 2 of C_T = 1e-5,
    worked out by hand above; the rationals there are re-checked here with
    exact arithmetic before the oracle's bits and betas are compared."""
    tau = abs(MARGINAL_BETA[0] - MARGINAL_BETA[2])
    assert tau == Fr(38, 3)
    for eps, g_hand, (lo, hi), bits_hand in MARGINAL_CASES:
        g = tuple(1 + tau / (b + eps) for b in MARGINAL_BETA)
        assert g == g_hand
        gam = [x ** 6 for x in g]
        chi = [x / sum(gam) for x in gam]
        assert lo < chi[2] < hi
        assert bits_hand == sum((0 if chi[k] < Fr(1, 10**5) else 1) << k for k in range(3))
        bits, beta = orc.face_bits(MARGINAL_W, float(eps), CT=1e-5)
        assert bits == bits_hand, (float(eps), bits)
        # beta_1 and beta_2 are exact in FP64; beta_0 = 9/4 + fl(13/12) is 10/3 to rounding
        assert abs(beta[0] - float(MARGINAL_BETA[0])) <= 2 * np.spacing(10.0 / 3.0)
        assert beta[1] == 1.0 and beta[2] == 16.0
    # the mirrored window moves the marginal stencil from 2 to 0
    bits, _ = orc.face_bits(MARGINAL_W[::-1], 1.0 / 8.0, CT=1e-5)
    assert bits == 0b110
