"""Pins of the oracle's Euler path: the Roe characteristic frame against the
analytic flux Jacobian, conservation, mirror symmetry of the '-' split, the
exact Riemann solutions of the Sod and Lax tubes (Sec. "Isolated wave
structure"), the exact Riemann solver itself, and the 2D dimension-by-dimension
form against the 1D scheme."""
import numpy as np
import pytest

from oracle import riemann
from paper_1808_00037_gb300 import inputs as I

G = 1.4


def jac_1d(U, g=G):
    rho, m, E = U
    u = m / rho
    p = (g - 1) * (E - 0.5 * rho * u * u)
    H = (E + p) / rho
    return np.array([[0, 1, 0],
                     [0.5 * (g - 3) * u * u, (3 - g) * u, g - 1],
                     [u * (0.5 * (g - 1) * u * u - H), H - (g - 1) * u * u, g * u]])


def flux_1d(U, g=G):
    rho, m, E = U
    u = m / rho
    p = (g - 1) * (E - 0.5 * rho * u * u)
    return np.array([m, m * u + p, u * (E + p)])


def roe_state_1d(UL, UR, g=G):
    def prim(U):
        rho, m, E = U
        u = m / rho
        p = (g - 1) * (E - 0.5 * rho * u * u)
        return rho, u, (E + p) / rho
    rl, ul, hl = prim(UL)
    rr, ur, hr = prim(UR)
    w = np.sqrt(rl) / (np.sqrt(rl) + np.sqrt(rr))
    u = w * ul + (1 - w) * ur
    H = w * hl + (1 - w) * hr
    rho = np.sqrt(rl * rr)
    return np.array([rho, rho * u, rho * H - (g - 1) / g * rho * (H - 0.5 * u * u)]), u, H


def test_frame_1d_eigensystem(orc):
    rng = np.random.default_rng(1)
    for _ in range(50):
        UL = I.prim_to_cons_1d(*rng.uniform([0.1, -2, 0.1], [3, 2, 10]))
        UR = I.prim_to_cons_1d(*rng.uniform([0.1, -2, 0.1], [3, 2, 10]))
        L, R, st = orc.frame_1d(UL, UR)
        assert st == 0
        assert np.allclose(L @ R, np.eye(3), atol=1e-12)
        Ut, u, H = roe_state_1d(UL, UR)
        A = jac_1d(Ut)
        c = np.sqrt((G - 1) * (H - 0.5 * u * u))
        lam = np.array([u - c, u, u + c])
        assert np.allclose(A @ R, R * lam[None, :], atol=1e-10 * (1 + np.abs(A).max()))
        # Roe's property: A(U~) (UR - UL) = F(UR) - F(UL)
        assert np.allclose(A @ (UR - UL), flux_1d(UR) - flux_1d(UL), atol=1e-10 * (1 + np.abs(A).max()))


def jac_2d_x(U, g=G):
    rho, mu, mv, E = U
    u, v = mu / rho, mv / rho
    q2 = 0.5 * (u * u + v * v)
    p = (g - 1) * (E - rho * q2)
    H = (E + p) / rho
    return np.array([[0, 1, 0, 0],
                     [(g - 1) * q2 - u * u, (3 - g) * u, -(g - 1) * v, g - 1],
                     [-u * v, v, u, 0],
                     [u * ((g - 1) * q2 - H), H - (g - 1) * u * u, -(g - 1) * u * v, g * u]])


def test_frame_2d_eigensystem(orc):
    rng = np.random.default_rng(2)
    for _ in range(30):
        for d in (0, 1):
            pl = rng.uniform([0.1, -1.2, -1.2, 0.03], [1.5, 1.2, 1.2, 1.5])
            pr = rng.uniform([0.1, -1.2, -1.2, 0.03], [1.5, 1.2, 1.2, 1.5])
            UL = I.prim_to_cons_2d(*pl)
            UR = I.prim_to_cons_2d(*pr)
            L, R, st = orc.frame_2d(UL, UR, d)
            assert st == 0
            assert np.allclose(L @ R, np.eye(4), atol=1e-12)
            # Roe state in the sweep direction; y is x with (u, v) swapped
            P = np.eye(4)[[0, 2, 1, 3]] if d == 1 else np.eye(4)
            wl = np.sqrt(pl[0]) / (np.sqrt(pl[0]) + np.sqrt(pr[0]))
            def Hof(pp):
                return (pp[3] / (G - 1) + 0.5 * pp[0] * (pp[1] ** 2 + pp[2] ** 2) + pp[3]) / pp[0]
            u = wl * pl[1] + (1 - wl) * pr[1]
            v = wl * pl[2] + (1 - wl) * pr[2]
            H = wl * Hof(pl) + (1 - wl) * Hof(pr)
            rho = np.sqrt(pl[0] * pr[0])
            p = (G - 1) / G * rho * (H - 0.5 * (u * u + v * v))
            Ut = I.prim_to_cons_2d(rho, u, v, p)
            A = P @ jac_2d_x(P @ Ut) @ P
            c = np.sqrt((G - 1) * (H - 0.5 * (u * u + v * v)))
            un = u if d == 0 else v
            lam = np.array([un - c, un, un, un + c])
            assert np.allclose(A @ R, R * lam[None, :], atol=1e-10 * (1 + np.abs(A).max()))


def test_euler_periodic_conservation_and_mirror(orc):
    n = 160
    x = (np.arange(n) + 0.5) / n
    rho = np.where((x > 0.3) & (x < 0.6), 1.0, 0.2) + 0.05 * np.sin(6 * np.pi * x)
    u = 0.3 + 0.2 * np.cos(2 * np.pi * x)
    p = np.where(x > 0.45, 2.0, 0.5)
    U = I.prim_to_cons_1d(rho, u, p)
    r, alpha, m = orc.rhs_1d(orc.SYS_EULER1D, U, 1.0 / n, want_masks=True)
    assert np.all(np.abs(r.sum(axis=1)) <= 1e-13 * np.abs(r).sum(axis=1))
    assert np.any(m != 0b11111)  # the jumps do switch stencils
    # reflection x -> 1 - x, u -> -u: RHS reflects, '+' <-> '-', field k <-> 2 - k
    Ur = I.prim_to_cons_1d(rho[::-1], -u[::-1], p[::-1])
    rr, alpha_r, mr = orc.rhs_1d(orc.SYS_EULER1D, Ur, 1.0 / n, want_masks=True)
    assert alpha_r == alpha
    sgn = np.array([1.0, -1.0, 1.0])[:, None]
    assert np.allclose(rr[:, ::-1] * sgn, r, rtol=0, atol=1e-11 * np.abs(r).max())
    for s in (0, 1):
        for k in range(3):
            assert np.array_equal(mr[1 - s, 2 - k][::-1], m[s, k])


def test_zero_gradient_flux_balance(orc):
    U, dx, x = I.riemann_tube(100, *I.SOD)
    r, _, _ = orc.rhs_1d(orc.SYS_EULER1D, U, dx, bc=(1, 1))
    # flat states at both ends: the boundary fluxes are the physical fluxes
    bal = flux_1d(U[:, 0]) - flux_1d(U[:, -1])
    assert np.allclose(r.sum(axis=1) * dx, bal, rtol=0, atol=1e-12)


@pytest.mark.parametrize("name,states,t_end,bound200", [("sod", I.SOD, 0.2, 5e-3), ("lax", I.LAX, 0.14, 1e-2)])
def test_shock_tubes_against_exact_riemann(orc, name, states, t_end, bound200):
    errs = []
    for n in (100, 200, 400):
        U, dx, x = I.riemann_tube(n, *states)
        Uf, steps, t, st = orc.run_1d(orc.SYS_EULER1D, U, dx, t_end=t_end, cfl=0.6, bc=(1, 1))
        assert st == 0 and t == pytest.approx(t_end, abs=1e-14)
        rho, u, p = riemann.sample(*states, (x - 0.5) / t_end)
        errs.append(np.mean(np.abs(Uf[0] - rho)))
        # no spurious oscillation beyond 1% of the exact solution's density range
        jump = rho.max() - rho.min()
        assert Uf[0].max() <= rho.max() + 0.01 * jump and Uf[0].min() >= rho.min() - 0.01 * jump
    assert errs[1] < bound200, errs
    assert errs[0] > errs[1] > errs[2], errs


def test_exact_riemann_solver_jump_conditions():
    for left, right in (I.SOD, I.LAX, ((1.0, -2.0, 0.4), (1.0, 2.0, 0.4)), ((1.0, 0.0, 1000.0), (1.0, 0.0, 0.01))):
        ps, us = riemann.star_state(left, right)
        smin, smax = riemann.wave_speeds(left, right)
        xi = np.linspace(smin - 1, smax + 1, 4001)
        rho, u, p = riemann.sample(left, right, xi)
        assert rho[0] == left[0] and rho[-1] == right[0]
        # the contact: p and u continuous across it
        k = np.searchsorted(xi, us)
        assert abs(p[k - 1] - ps) < 1e-10 * ps and abs(p[k] - ps) < 1e-10 * ps
        # Rankine-Hugoniot across each shock (shock speed = Lax-jump location)
        for side, (rk, uk, pk) in (("L", left), ("R", right)):
            if ps > pk:
                S = smin if side == "L" else smax
                rs = rho[k - 1] if side == "L" else rho[k]
                m0, m1 = rk * (uk - S), rs * (us - S)
                assert abs(m0 - m1) < 1e-9 * abs(m0)
                assert abs((m0 * uk + pk) - (m1 * us + ps)) < 1e-9 * (abs(m0 * uk) + pk)
    # symmetric double rarefaction: closed form p* = p (1 - (g-1) u / (2c))^(2g/(g-1))
    c = np.sqrt(G * 0.4 / 1.0)
    ps, us = riemann.star_state((1.0, -0.3, 0.4), (1.0, 0.3, 0.4))
    assert abs(ps - 0.4 * (1 - (G - 1) * 0.3 / (2 * c)) ** (2 * G / (G - 1))) < 1e-12 and abs(us) < 1e-14


def test_2d_reduces_to_1d(orc):
    """y-independent data with v = 0: the 2D RHS equals the 1D Euler RHS on
    (rho, rho u, E) and vanishes on rho v."""
    n, ny = 64, 9
    x = (np.arange(n) + 0.5) / n
    rho = np.where(x < 0.4, 1.0, 0.3) + 0.02 * np.sin(2 * np.pi * x)
    u = 0.2 * np.cos(2 * np.pi * x)
    p = np.where(x < 0.55, 1.0, 0.2)
    U1 = I.prim_to_cons_1d(rho, u, p)
    r1, a1, _ = orc.rhs_1d(orc.SYS_EULER1D, U1, 1.0 / n)
    U2 = np.zeros((4, ny, n))
    U2[0], U2[1], U2[3] = U1[0], U1[1], U1[2]
    r2, (ax, ay), _ = orc.rhs_2d(U2, 1.0 / n, 1.0 / ny, bc=(0, 0, 0, 0))
    assert ax == a1
    assert np.all(r2[2] == 0.0)
    for c1, c2 in ((0, 0), (1, 1), (2, 3)):
        assert np.allclose(r2[c2], r1[c1][None, :], rtol=0, atol=1e-12 * np.abs(r1[c1]).max())


def test_2d_transpose_symmetry_and_conservation(orc):
    U, dx, dy, _ = I.quadrants_2d(4, 24, 24)
    U = U + 0.01 * np.sin(np.arange(24))[None, None, :]
    r, (ax, ay), _ = orc.rhs_2d(U, dx, dy, bc=(0, 0, 0, 0))
    assert np.all(np.abs(r.sum(axis=(1, 2))) <= 1e-12 * np.abs(r).sum(axis=(1, 2)))
    Ut = np.stack([U[0].T, U[2].T, U[1].T, U[3].T])
    rt, (axt, ayt), _ = orc.rhs_2d(Ut, dy, dx, bc=(0, 0, 0, 0))
    assert axt == ay and ayt == ax
    back = np.stack([rt[0].T, rt[2].T, rt[1].T, rt[3].T])
    assert np.allclose(back, r, rtol=0, atol=1e-11 * np.abs(r).max())


def test_2d_uniform_steady(orc):
    U = I.prim_to_cons_2d(np.full((5, 7), 0.8), np.full((5, 7), 0.3), np.full((5, 7), -0.2), np.full((5, 7), 1.1))
    for bc in ((0, 0, 0, 0), (1, 1, 1, 1)):
        r, _, _ = orc.rhs_2d(U, 0.1, 0.1, bc=bc)
        assert np.all(r == 0.0)


def test_shu_osher_self_convergence(orc):
    """Shu-Osher has no exact solution (the paper compares with a fine WENO-JS
    run); the oracle's own solutions at N = 200, 400, 800 to t = 1.8 approach
    its N = 1600 solution (sampled at the coarse cell centres), each doubling
    at least halving the mean density error."""
    sols = {}
    for n in (200, 400, 800, 1600):
        U, dx = I.shu_osher(n)
        Uf, _, t, st = orc.run_1d(orc.SYS_EULER1D, U, dx, t_end=1.8, cfl=0.5, bc=(1, 1))
        assert st == 0 and t == 1.8
        sols[n] = Uf[0]
    errs = []
    for n in (200, 400, 800):
        r = 1600 // n
        f = sols[1600].reshape(n, r)
        errs.append(np.abs(sols[n] - 0.5 * (f[:, r // 2 - 1] + f[:, r // 2])).mean())
    assert errs[1] < 0.5 * errs[0] and errs[2] < 0.5 * errs[1], errs


def isentropic_vortex(x, y, eps=5.0, g=G, x0=5.0, y0=5.0):
    """Conserved variables of the isentropic vortex in the mean flow
    (rho, u, v, p) = (1, 1, 1, 1): an exact smooth solution of the 2D Euler
    equations that translates with velocity (1, 1).  Analytic in x and y, so
    complex arguments give exact derivatives by the complex step."""
    ex, ey = x - x0, y - y0
    f = np.exp(0.5 * (1 - (ex * ex + ey * ey)))
    u = 1 - eps / (2 * np.pi) * f * ey
    v = 1 + eps / (2 * np.pi) * f * ex
    T = 1 - (g - 1) * eps**2 / (8 * g * np.pi**2) * f * f
    rho = T ** (1 / (g - 1))
    p = rho * T
    return np.stack([rho, rho * u, rho * v, p / (g - 1) + 0.5 * rho * (u * u + v * v)])


def test_2d_order_on_the_isentropic_vortex(orc):
    """The 2D right-hand side against the exact time derivative of the
    translating vortex, -(dU/dx + dU/dy) (complex-step derivatives of the
    closed form), on [0, 10]^2 with N = 80, 160, 320: every stencil is kept in
    the vortex core (the linear seventh-order scheme in both sweeps) and the
    maximum error there falls at order 6.8-7.0 (the periodic wrap of the
    not-quite-periodic tails, ~4e-6, is outside the core)."""
    errs = []
    for n in (80, 160, 320):
        d = 10.0 / n
        c = (np.arange(n) + 0.5) * d
        X, Y = np.meshgrid(c, c)  # [ny, nx]
        U = isentropic_vortex(X, Y)
        h = 1e-30
        exact = -(isentropic_vortex(X + 1j * h, Y).imag + isentropic_vortex(X, Y + 1j * h).imag) / h
        r, _, (xm, ym) = orc.rhs_2d(U, d, d, bc=(0, 0, 0, 0), want_masks=True)
        core = (np.abs(X - 5) < 2.5) & (np.abs(Y - 5) < 2.5)
        rows, cols = core.any(axis=1), core.any(axis=0)  # xm is [.., y, face], ym [.., x, face]
        assert np.all(xm[:, :, rows, :] == 31) and np.all(ym[:, :, cols, :] == 31)
        errs.append(np.abs(r - exact)[:, core].max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 6.6) and orders[-1] > 6.85 and np.all(orders < 7.3), orders


def test_1d_euler_order_on_an_entropy_wave(orc):
    """rho = 1 + 0.2 sin(2 pi x), u = p = 1 on a periodic [0, 1): an exact
    solution that translates with speed 1, so L(U) = -(rho', rho', rho'/2)
    exactly.  Every stencil of every field is kept and the maximum error falls
    at order ~7 (N = 20, 40, 80; at N = 160 it nears FP64 round-off)."""
    errs = []
    for n in (20, 40, 80):
        x = (np.arange(n) + 0.5) / n
        U = I.prim_to_cons_1d(1 + 0.2 * np.sin(2 * np.pi * x), np.ones(n), np.ones(n))
        dr = 0.4 * np.pi * np.cos(2 * np.pi * x)
        r, _, m = orc.rhs_1d(orc.SYS_EULER1D, U, 1.0 / n, want_masks=True)
        assert np.all(m == 31)
        errs.append(np.abs(r + np.stack([dr, dr, 0.5 * dr])).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 6.9) and np.all(orders < 7.1), orders
