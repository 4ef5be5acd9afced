"""Pins of the oracle's per-field Lax-Friedrichs alpha (the alpha switch,
oracle.alpha_mode(ALPHA_PER_FIELD)): alpha_k = max_i |lambda_k(U_i)| per
characteristic field (1D Euler: u - c, u, u + c), and each field's split
values (L_k F +- alpha_k L_k U) / 2 in the face's Roe frame.  The paper uses
one global alpha (Sec. "One dimensional Euler equations"); the per-field form
is the option of the boundary's alpha mode.  These checks rest on facts fixed
by the mathematics, not on the oracle's own expressions:
  - the per-field maxima are those of |u - c|, |u|, |u + c| (computed here
    from the primitive variables), and their maximum is the global alpha;
  - with every field's alpha equal to the global one the split values equal
    the global split's L_k (F +- alpha U)/2 (linearity of L_k), so the RHS
    agrees with the global-alpha RHS to round-off;
  - the RHS stays conservative (periodic sums vanish);
  - on an entropy wave (u and p constant, rho varying) the entropy field's
    row of L annihilates (0, p, u p), so L_1 F = u L_1 U and the split value
    of the entropy field against the flow vanishes exactly when alpha_1 = |u|:
    a per-field alpha of the wrong field, or the global alpha, leaves it finite;
  - a scalar law has one field, so both alpha modes coincide bit for bit."""
import numpy as np

import oracle
from paper_1808_00037_gb300 import inputs as I

E1 = oracle.SYS_EULER1D
G = 1.4


def _prims(U):
    rho, mu, E = U
    u = mu / rho
    p = (G - 1.0) * (E - 0.5 * mu * u)
    return rho, u, p


def _entropy_wave(n, u, seed=3):
    rng = np.random.default_rng(seed)
    x = (np.arange(n) + 0.5) / n
    rho = 1.0 + 0.3 * np.sin(2 * np.pi * x) + 0.1 * rng.uniform(-1, 1) * np.cos(6 * np.pi * x)
    p = np.full(n, 1.0)
    uu = np.full(n, u)
    return I.prim_to_cons_1d(rho, uu, p), 1.0 / n


def test_per_field_alphas_are_the_eigenvalue_maxima():
    for seed in (9, 10, 11):
        U, dx, _ = I.random_euler_smooth(seed, 301)
        rho, u, p = _prims(U)
        c = np.sqrt(G * p / rho)
        want = [np.max(np.abs(u - c)), np.max(np.abs(u)), np.max(np.abs(u + c))]
        got = oracle.alpha_fields_1d(E1, U)
        assert np.allclose(got, want, rtol=1e-14, atol=0)
        assert got.max() == oracle.alpha_1d(E1, U)
    U, dx = I.shu_osher(400)
    assert oracle.alpha_fields_1d(E1, U).max() == oracle.alpha_1d(E1, U)


def test_equal_field_alphas_reduce_to_the_global_split():
    for U, dx, bc in ((I.shu_osher(400)[0], I.shu_osher(400)[1], (1, 1)),
                      (*I.random_euler_smooth(9, 257)[:2], (0, 0)),
                      (*I.riemann_tube(203, *I.SOD)[:2], (1, 1))):
        a = oracle.alpha_1d(E1, U)
        L0, _, m0 = oracle.rhs_1d(E1, U, dx, bc=bc, alpha=a, want_masks=True)
        faces = (-1, 17, U.shape[1] // 2)
        P0 = [oracle.face_split_1d(E1, U, i, bc=bc, alpha=a) for i in faces]
        with oracle.alpha_mode(oracle.ALPHA_PER_FIELD):
            L1, _, m1 = oracle.rhs_1d(E1, U, dx, bc=bc, alpha=a, want_masks=True)
            P1 = [oracle.face_split_1d(E1, U, i, bc=bc, alpha=a) for i in faces]
        for (p0, q0), (p1, q1) in zip(P0, P1):
            s = max(np.abs(p0).max(), np.abs(q0).max())
            assert np.abs(p1 - p0).max() <= 1e-13 * s and np.abs(q1 - q0).max() <= 1e-13 * s
        scale = np.abs(L0).max()
        assert np.abs(L1 - L0).max() <= 1e-12 * scale
        assert (m1 == m0).mean() >= 0.999


def test_per_field_rhs_is_conservative():
    U, dx, _ = I.random_euler_smooth(12, 320)
    with oracle.alpha_mode(oracle.ALPHA_PER_FIELD):
        L, _, _ = oracle.rhs_1d(E1, U, dx, bc=(0, 0))
    assert np.all(np.abs(L.sum(axis=1)) <= 1e-11 * np.abs(L).max() * L.shape[1])


def test_entropy_field_split_against_the_flow_vanishes():
    for u in (0.4, -0.4):
        U, dx = _entropy_wave(200, u)
        against = 1 if u > 0 else 0  # the split carrying information against the flow
        for i in (-1, 50, 123):
            with oracle.alpha_mode(oracle.ALPHA_PER_FIELD):
                Pp, Pm = oracle.face_split_1d(E1, U, i)
            P = (Pp, Pm)
            scale = np.abs(P[1 - against][1]).max()
            assert scale > 1e-2
            assert np.abs(P[against][1]).max() <= 1e-13 * scale, (u, i)
            # the acoustic fields' splits stay finite both ways
            assert np.abs(P[against][0]).max() > 1e-3 and np.abs(P[against][2]).max() > 1e-3
            # with the global alpha the entropy field's split against the flow does not vanish
            Gp, Gm = oracle.face_split_1d(E1, U, i)
            assert np.abs((Gp, Gm)[against][1]).max() > 1e-3 * scale


def test_scalar_laws_have_one_mode():
    for sysid, U, dx in ((oracle.SYS_ADVECTION, *I.advection_sine(160)[:2]),
                         (oracle.SYS_BURGERS, *I.burgers_sine(160)[:2])):
        L0, _, m0 = oracle.rhs_1d(sysid, U, dx, want_masks=True)
        with oracle.alpha_mode(oracle.ALPHA_PER_FIELD):
            L1, _, m1 = oracle.rhs_1d(sysid, U, dx, want_masks=True)
        assert np.array_equal(L0, L1) and np.array_equal(m0, m1)


def test_per_field_run_conserves_and_stays_physical():
    U, dx, _ = I.random_euler_smooth(9, 257)
    with oracle.alpha_mode(oracle.ALPHA_PER_FIELD):
        Uo, steps, t, st = oracle.run_1d(E1, U, dx, t_end=0.05, cfl=0.5, bc=(0, 0))
    assert st == oracle.OK and steps > 0
    s0, s1 = U.sum(axis=1), Uo.sum(axis=1)
    assert np.allclose(s0, s1, rtol=1e-13, atol=0)
    rho, u, p = _prims(Uo)
    assert np.all(rho > 0) and np.all(p > 0)
