"""Seeded, synthetic initial data for the TENO7-ext workloads.

This module holds initial conditions only -- no step of the scheme -- so the
CUDA path and the CPU oracle can both be fed from it.  Every generator returns
float64 numpy arrays of conserved variables, variable-major: [m, n] in 1D and
[4, ny, nx] in 2D, sampled at cell centres x_i = x0 + (i + 1/2) dx (point
values of the finite-difference form, Eq. dis).
"""
from __future__ import annotations

import numpy as np

GAMMA = 1.4


def cell_centres(x0: float, x1: float, n: int) -> tuple[np.ndarray, float]:
    dx = (x1 - x0) / n
    return x0 + (np.arange(n) + 0.5) * dx, dx


def prim_to_cons_1d(rho, u, p, gamma=GAMMA) -> np.ndarray:
    rho = np.asarray(rho, np.float64)
    u = np.asarray(u, np.float64)
    p = np.asarray(p, np.float64)
    return np.stack([rho, rho * u, p / (gamma - 1.0) + 0.5 * rho * u * u])


def cons_to_prim_1d(U, gamma=GAMMA):
    rho = U[0]
    u = U[1] / rho
    p = (gamma - 1.0) * (U[2] - 0.5 * U[1] * u)
    return rho, u, p


def prim_to_cons_2d(rho, u, v, p, gamma=GAMMA) -> np.ndarray:
    return np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


# ------------------------------------------------------------ scalar ------
def advection_sine(n: int, x0=-1.0, x1=1.0):
    """u0 = sin(pi x) on [-1, 1], periodic (advection accuracy case)."""
    x, dx = cell_centres(x0, x1, n)
    return np.sin(np.pi * x)[None, :], dx, x


def advection_gaussian(n: int):
    """u1 = exp(-300 (x - 0.5)^2) on [0, 1) (Eq. init_LinAdv)."""
    x, dx = cell_centres(0.0, 1.0, n)
    return np.exp(-300.0 * (x - 0.5) ** 2)[None, :], dx, x


def advection_sin3(n: int):
    """u2 = sin(pi x)^3 on [0, 2) (Eq. init_LinAdv2), second-order critical points."""
    x, dx = cell_centres(0.0, 2.0, n)
    return (np.sin(np.pi * x) ** 3)[None, :], dx, x


def four_wave(n: int = 400):
    """u3 of Eq. init_LinAdv3 on [-1, 1), periodic: Gaussian, square wave,
    triangle and half ellipse (Eqs. FG, coof).  The printed intervals lie in
    [0.2, 1.6], outside the stated domain, and the triangle printed there is
    negative; they are read as shifted by +1, i.e. the pieces sit on
    [-0.8, -0.6], [-0.4, -0.2], [0, 0.2] and [0.4, 0.6], with the Gaussian
    centre z = -0.7 (printed 0.7), the triangle 1 - |10 (x - 0.1)| and the
    ellipse centre a = 0.5 as printed."""
    x, dx = cell_centres(-1.0, 1.0, n)
    z, delta, alpha, a = -0.7, 0.005, 10.0, 0.5
    beta = np.log(2.0) / (36.0 * delta * delta)

    def G(xx, zz):
        return np.exp(-beta * (xx - zz) ** 2)

    def F(xx, aa):
        return np.sqrt(np.maximum(1.0 - alpha * alpha * (xx - aa) ** 2, 0.0))

    u = np.zeros(n)
    m = (x >= -0.8) & (x <= -0.6)
    u[m] = (G(x[m], z - delta) + G(x[m], z + delta) + 4.0 * G(x[m], z)) / 6.0
    m = (x >= -0.4) & (x <= -0.2)
    u[m] = 1.0
    m = (x >= 0.0) & (x <= 0.2)
    u[m] = 1.0 - np.abs(10.0 * (x[m] - 0.1))
    m = (x >= 0.4) & (x <= 0.6)
    u[m] = (F(x[m], a - delta) + F(x[m], a + delta) + 4.0 * F(x[m], a)) / 6.0
    return u[None, :], dx, x


def burgers_sine(n: int):
    """u = 1/2 + sin(pi x) on [0, 2) (inviscid Burgers case)."""
    x, dx = cell_centres(0.0, 2.0, n)
    return (0.5 + np.sin(np.pi * x))[None, :], dx, x


def random_smooth_1d(seed: int, n: int, modes: int = 6, amp: float = 0.3):
    """Random periodic trigonometric data on [0, 1): a smooth, seeded scalar field."""
    rng = np.random.default_rng(seed)
    x, dx = cell_centres(0.0, 1.0, n)
    u = np.zeros(n)
    for k in range(1, modes + 1):
        a, b = rng.normal(0.0, amp / k, 2)
        u += a * np.sin(2 * np.pi * k * x) + b * np.cos(2 * np.pi * k * x)
    return u[None, :], dx, x


# ------------------------------------------------------------- Euler 1D ----
SHU_OSHER_LEFT = (3.857143, 2.629369, 10.33333)


def shu_osher(n: int = 1600, tiles: int = 1):
    """Shu-Osher shock / entropy-wave interaction on [-5, 5]: left state for
    x < -4, right state (1 + 0.2 sin 5x, 0, 1).  ``tiles`` > 1 repeats the
    profile end to end (same dx, n cells per copy) to build a long domain with
    the same local structure."""
    x, dx = cell_centres(-5.0, 5.0, n)
    rho = np.where(x < -4.0, SHU_OSHER_LEFT[0], 1.0 + 0.2 * np.sin(5.0 * x))
    u = np.where(x < -4.0, SHU_OSHER_LEFT[1], 0.0)
    p = np.where(x < -4.0, SHU_OSHER_LEFT[2], 1.0)
    U = prim_to_cons_1d(rho, u, p)
    if tiles > 1:
        U = np.tile(U, (1, tiles))
    return U, dx


def riemann_tube(n: int, left, right, x0=0.0, x1=1.0, xd=0.5):
    """Piecewise-constant Riemann data (rho, u, p), discontinuity at xd."""
    x, dx = cell_centres(x0, x1, n)
    pick = x < xd
    rho = np.where(pick, left[0], right[0])
    u = np.where(pick, left[1], right[1])
    p = np.where(pick, left[2], right[2])
    return prim_to_cons_1d(rho, u, p), dx, x


SOD = ((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
LAX = ((0.445, 0.698, 3.528), (0.5, 0.0, 0.571))


def titarev_toro(n: int = 400):
    x, dx = cell_centres(0.0, 10.0, n)
    left = x <= 0.5
    rho = np.where(left, 1.515695, 1.0 + 0.1 * np.sin(20.0 * np.pi * x))
    u = np.where(left, 0.523346, 0.0)
    p = np.where(left, 1.80500, 1.0)
    return prim_to_cons_1d(rho, u, p), dx, x


def random_euler_smooth(seed: int, n: int):
    """Smooth periodic Euler state on [0, 1) with positive density and pressure."""
    rng = np.random.default_rng(seed)
    x, dx = cell_centres(0.0, 1.0, n)
    a = rng.uniform(-0.2, 0.2, 3)
    ph = rng.uniform(0, 2 * np.pi, 3)
    rho = 1.0 + a[0] * np.sin(2 * np.pi * x + ph[0])
    u = 0.5 + a[1] * np.sin(4 * np.pi * x + ph[1])
    p = 1.0 + a[2] * np.sin(2 * np.pi * x + ph[2])
    return prim_to_cons_1d(rho, u, p), dx, x


# --------------------------------------------------- batched Riemann tubes --
def riemann_tube_batch(seed: int, ntubes: int = 4096, nmin: int = 256, nmax: int = 8192):
    """Ragged batch of independent Riemann tubes on [0, 1], discontinuity at 0.5.
    Lengths ~ U[nmin, nmax]; left/right states rho ~ U[0.1, 2], u ~ U[-1, 1],
    p ~ U[0.1, 10].  Returns (U_concat[3, sum n], offsets[ntubes+1], dx[ntubes], states)."""
    rng = np.random.default_rng(seed)
    lengths = rng.integers(nmin, nmax + 1, size=ntubes)
    states = np.empty((ntubes, 2, 3))
    states[:, :, 0] = rng.uniform(0.1, 2.0, (ntubes, 2))
    states[:, :, 1] = rng.uniform(-1.0, 1.0, (ntubes, 2))
    states[:, :, 2] = rng.uniform(0.1, 10.0, (ntubes, 2))
    offsets = np.zeros(ntubes + 1, np.int64)
    offsets[1:] = np.cumsum(lengths)
    U = np.empty((3, int(offsets[-1])))
    dx = np.empty(ntubes)
    for t in range(ntubes):
        Ut, dxt, _ = riemann_tube(int(lengths[t]), tuple(states[t, 0]), tuple(states[t, 1]))
        U[:, offsets[t]:offsets[t + 1]] = Ut
        dx[t] = dxt
    return U, offsets, dx, states


# -------------------------------------------------------------- 2D Euler ----
def quadrants_2d(seed: int, nx: int = 2048, ny: int = 2048, max_tries: int = 1000):
    """Four-quadrant Riemann data on [0, 1]^2 with per-quadrant (rho, u, v, p):
    rho ~ U[0.1, 1.5], p ~ U[0.03, 1.5], u, v ~ U[-1.2, 1.2].  Draws whose
    neighbouring quadrants would open a vacuum (normal velocity jump >= 5 x the
    sum of the sound speeds) are redrawn.  Returns (U[4, ny, nx], dx, dy, states)."""
    rng = np.random.default_rng(seed)
    g = GAMMA
    for _ in range(max_tries):
        rho = rng.uniform(0.1, 1.5, 4)
        p = rng.uniform(0.03, 1.5, 4)
        u = rng.uniform(-1.2, 1.2, 4)
        v = rng.uniform(-1.2, 1.2, 4)
        c = np.sqrt(g * p / rho)
        # quadrants: 0 = (x>.5,y>.5), 1 = (x<.5,y>.5), 2 = (x<.5,y<.5), 3 = (x>.5,y<.5)
        ok = True
        for a, b, vel in ((1, 0, u), (2, 3, u), (3, 0, v), (2, 1, v)):
            if vel[b] - vel[a] >= 5.0 * (c[a] + c[b]):
                ok = False
        if ok:
            break
    xs, dx = cell_centres(0.0, 1.0, nx)
    ys, dy = cell_centres(0.0, 1.0, ny)
    X, Y = np.meshgrid(xs, ys)
    q = np.where(X > 0.5, np.where(Y > 0.5, 0, 3), np.where(Y > 0.5, 1, 2))
    U = prim_to_cons_2d(rho[q], u[q], v[q], p[q])
    return U, dx, dy, np.stack([rho, u, v, p], axis=1)


def random_smooth_2d(seed: int, nx: int, ny: int):
    """Smooth periodic 2D Euler state on [0, 1)^2."""
    rng = np.random.default_rng(seed)
    xs, dx = cell_centres(0.0, 1.0, nx)
    ys, dy = cell_centres(0.0, 1.0, ny)
    X, Y = np.meshgrid(xs, ys)
    a = rng.uniform(-0.2, 0.2, 4)
    rho = 1.0 + a[0] * np.sin(2 * np.pi * (X + Y))
    u = 0.4 + a[1] * np.cos(2 * np.pi * Y)
    v = -0.3 + a[2] * np.sin(2 * np.pi * X)
    p = 1.0 + a[3] * np.cos(2 * np.pi * (X - Y))
    return prim_to_cons_2d(rho, u, v, p), dx, dy


# --------------------------------------------------------------- adjoint ----
def adjoint_modes(seed: int, K: int = 64):
    """a_k ~ N(0, (0.02/k)^2), k = 1..K."""
    rng = np.random.default_rng(seed)
    k = np.arange(1, K + 1)
    return rng.normal(0.0, 1.0, K) * (0.02 / k)


def adjoint_ic(a_k: np.ndarray, n: int = 4096):
    """rho0 = 1 + sum_k a_k sin(2 pi k x), u0 = 1, p0 = 1 on periodic [0, 1)."""
    x, dx = cell_centres(0.0, 1.0, n)
    k = np.arange(1, a_k.size + 1)
    rho = 1.0 + np.sin(2 * np.pi * np.outer(x, k)) @ a_k
    return prim_to_cons_1d(rho, np.ones(n), np.ones(n)), dx, x
