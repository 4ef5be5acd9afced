"""The hand-written discrete adjoint (t7_euler_rhs_adjoint, t7_rk3_step_adjoint,
and the checkpointed autograd Function) against finite differences:

* dot-product test of the RHS adjoint against central differences of the
  ORACLE's right-hand side with alpha held at alpha(U) (the adjoint freezes
  alpha and the stencil selection; the perturbation is small enough that the
  oracle's masks do not change, which the test checks);
* dot-product test of one RK3 step's adjoint against GPU forward differences;
* gradients of J = sum rho^2 dx for the sine-mode problem against central
  differences of the oracle (reduced size) and of the GPU forward (full size:
  N = 4096, 2000 steps, checkpoints every 100 steps);
* dot-product tests of the RHS adjoint, the RK3-step adjoint and the reduced
  sine-mode gradient against the oracle's tangent-linear mode (the exact
  directional derivative with the same frozen selection and alpha) in FP64
  to 1e-10.
"""
import numpy as np
import pytest

import oracle
from paper_1808_00037_gb300 import adjoint as A
from paper_1808_00037_gb300 import binding as B
from paper_1808_00037_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def states():
    yield "smooth", I.random_euler_smooth(2, 300)[:2], (0, 0)
    U, dx, _ = I.riemann_tube(300, *I.SOD)
    yield "sod", (U, dx), (1, 1)
    U, dx = I.shu_osher(400)
    yield "shu-osher", (U, dx), (1, 1)


@pytest.mark.parametrize("prec", [B.T7_F64, B.T7_F32])
def test_rhs_adjoint_dot_product_against_oracle_fd(prec):
    rng = np.random.default_rng(5)
    for name, (U, dx), bc in states():
        n = U.shape[1]
        _, alpha, m0 = oracle.rhs_1d(oracle.SYS_EULER1D, U, dx, bc=bc, want_masks=True)
        v = rng.normal(size=U.shape)
        w = rng.normal(size=U.shape) * np.abs(U)
        # fourth-order central difference: accurate to ~1e-10 relative here
        # (h and 2h agree to that), the selection unchanged at +-h and +-2h
        h = 1e-5
        r = {}
        for s in (1, -1, 2, -2):
            r[s], _, ms = oracle.rhs_1d(oracle.SYS_EULER1D, U + s * h * w, dx, bc=bc, alpha=alpha, want_masks=True)
            assert np.array_equal(ms, m0), (name, s)  # selection frozen
        lhs = np.sum(v * (8 * (r[1] - r[-1]) - (r[2] - r[-2])) / (12 * h))
        dtype = torch.float64 if prec == B.T7_F64 else torch.float32
        c = B.Context(B.T7_EULER1D, n, dx, prec=prec, bc=(bc[0], bc[1], 0, 0))
        out = c.euler_rhs_adjoint(torch.tensor(U, dtype=dtype, device="cuda"),
                                  torch.tensor(v, dtype=dtype, device="cuda"))
        c.sync()
        rhs = np.sum(out.double().cpu().numpy() * w)
        tol = 1e-8 if prec == B.T7_F64 else 2e-3
        assert abs(lhs - rhs) <= tol * max(abs(lhs), 1e-12), (name, lhs, rhs)


def test_rk3_step_adjoint_dot_product():
    """<lambda, dS(U) w> (central differences of the GPU step, fixed dt) equals
    <S^T lambda, w> on smooth periodic data (alpha's variation is below the
    difference tolerance there)."""
    rng = np.random.default_rng(8)
    U, dx, _ = I.random_euler_smooth(4, 512)
    c = B.Context(B.T7_EULER1D, 512, dx, bc=(0, 0, 0, 0))
    Ud = torch.tensor(U, device="cuda")
    dt = c.cfl_dt(Ud, 0.5)
    lam = rng.normal(size=U.shape)
    w = rng.normal(size=U.shape) * np.abs(U)
    h = 1e-6
    out = []
    for sgn in (1, -1):
        X = torch.tensor(U + sgn * h * w, device="cuda")
        c.rk3_step(X, dt)
        c.sync()
        out.append(X.cpu().numpy())
    lhs = np.sum(lam * (out[0] - out[1]) / (2 * h))
    L = torch.tensor(lam, device="cuda")
    c.rk3_step_adjoint(Ud, dt, L)
    c.sync()
    rhs = np.sum(L.cpu().numpy() * w)
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs), (lhs, rhs)


def _oracle_J(a, n, nsteps, dt):
    U0, dx, _ = I.adjoint_ic(a, n)
    Uf, s, t, st = oracle.run_1d(oracle.SYS_EULER1D, U0, dx, t_end=np.inf, dt_fixed=dt, max_steps=nsteps,
                                 bc=(0, 0))
    assert s == nsteps and st == 0
    return float(np.sum(Uf[0] ** 2) * dx)


def test_sine_mode_gradient_reduced_against_oracle_fd():
    a = I.adjoint_modes(3, K=8)
    n, nsteps = 256, 200
    J, g, dt = A.sine_modes_gradient(a, n=n, nsteps=nsteps, every=20)
    assert J == pytest.approx(_oracle_J(a, n, nsteps, dt), rel=1e-12)
    for k in range(8):
        h = 1e-5 * max(abs(a[k]), 1e-3)
        ap, am = a.copy(), a.copy()
        ap[k] += h
        am[k] -= h
        fd = (_oracle_J(ap, n, nsteps, dt) - _oracle_J(am, n, nsteps, dt)) / (2 * h)
        assert abs(g[k] - fd) <= 1e-6 * np.max(np.abs(g)) + 1e-6 * abs(fd), (k, g[k], fd)


@pytest.mark.parametrize("prec", [B.T7_F64, B.T7_F32])
def test_sine_mode_gradient_full_config(prec):
    """N = 4096, 2000 steps, 64 modes, checkpoints every 100 steps: the adjoint
    gradient matches central differences of the GPU FP64 forward on a spread
    of modes (FP64 to 1e-6, FP32 to 2e-3 of the gradient's scale)."""
    a = I.adjoint_modes(11, K=64)
    J, g, dt = A.sine_modes_gradient(a, n=4096, nsteps=2000, every=100, prec=prec)
    scale = np.max(np.abs(g))
    for k in (0, 1, 7, 31, 63):
        h = 1e-6
        ap, am = a.copy(), a.copy()
        ap[k] += h
        am[k] -= h
        fd = (A.sine_modes_objective(ap, 4096, 2000, dt) - A.sine_modes_objective(am, 4096, 2000, dt)) / (2 * h)
        tol = 1e-6 if prec == B.T7_F64 else 2e-3
        assert abs(g[k] - fd) <= tol * scale, (k, g[k], fd, scale)


@pytest.mark.parametrize("prec", [B.T7_F64, B.T7_F32])
def test_recorded_step_and_its_adjoint(prec):
    """t7_rk3_step_record advances exactly like t7_rk3_step (bit for bit), and
    t7_rk3_step_adjoint_recorded gives the same map as t7_rk3_step_adjoint
    (FP64 to 1e-12, FP32 to 1e-4 of the result's scale; the two differ in
    summation order only), on smooth periodic data and on Shu-Osher."""
    dtype = torch.float64 if prec == B.T7_F64 else torch.float32
    rng = np.random.default_rng(21)
    for (U, dx), bc in ((I.random_euler_smooth(4, 512)[:2], (0, 0)), (I.shu_osher(400), (1, 1))):
        n = U.shape[1]
        c = B.Context(B.T7_EULER1D, n, dx, prec=prec, bc=(bc[0], bc[1], 0, 0))
        Ud = torch.tensor(U, dtype=dtype, device="cuda")
        dt = c.cfl_dt(Ud, 0.5)
        ref = Ud.clone()
        c.rk3_step(ref, dt)
        tape = torch.zeros(c.tape_bytes(), dtype=torch.uint8, device="cuda")
        out = torch.empty_like(Ud)
        c.rk3_step_record(Ud, out, dt, tape)
        c.sync()
        assert torch.equal(out, ref)
        lam = torch.tensor(rng.normal(size=U.shape), dtype=dtype, device="cuda")
        l_old = lam.clone()
        c.rk3_step_adjoint(Ud, dt, l_old)
        l_new = lam.clone()
        c.rk3_step_adjoint_recorded(Ud, tape, dt, l_new)
        c.sync()
        scale = float(l_old.abs().max())
        tol = 1e-12 if prec == B.T7_F64 else 1e-4
        assert float((l_new - l_old).abs().max()) <= tol * scale


# ---- against the oracle's tangent-linear mode (forward-mode derivative with
# the same frozen selection and alpha), by the dot-product identity
# <v, J u> = <J^T v, u>, in FP64 to 1e-10

def test_rhs_adjoint_dot_product_against_tangent_linear_oracle():
    rng = np.random.default_rng(15)
    for name, (U, dx), bc in states():
        n = U.shape[1]
        _, alpha, masks = oracle.rhs_1d(oracle.SYS_EULER1D, U, dx, bc=bc, want_masks=True)
        v = rng.normal(size=U.shape)
        u = rng.normal(size=U.shape) * np.abs(U)
        _, Ju = oracle.rhs_1d_tl(oracle.SYS_EULER1D, U, u, dx, alpha, masks, bc=bc)
        lhs = np.sum(v * Ju)
        c = B.Context(B.T7_EULER1D, n, dx, prec=B.T7_F64, bc=(bc[0], bc[1], 0, 0))
        out = c.euler_rhs_adjoint(torch.tensor(U, device="cuda"), torch.tensor(v, device="cuda"))
        c.sync()
        rhs = np.sum(out.cpu().numpy() * u)
        assert abs(lhs - rhs) <= 1e-10 * abs(lhs), (name, lhs, rhs)
        c.close()


def test_rk3_step_adjoint_dot_product_against_tangent_linear_oracle():
    """One step's adjoint (stage alphas and selections frozen at the primal
    stage states) on smooth periodic data and on Shu-Osher."""
    rng = np.random.default_rng(16)
    for (U, dx), bc in ((I.random_euler_smooth(4, 512)[:2], (0, 0)), (I.shu_osher(400), (1, 1))):
        n = U.shape[1]
        c = B.Context(B.T7_EULER1D, n, dx, prec=B.T7_F64, bc=(bc[0], bc[1], 0, 0))
        Ud = torch.tensor(U, device="cuda")
        dt = c.cfl_dt(Ud, 0.5)
        lam = rng.normal(size=U.shape)
        w = rng.normal(size=U.shape) * np.abs(U)
        _, Sw = oracle.rk3_step_1d_tl(oracle.SYS_EULER1D, U, w, dx, dt, bc=bc)
        lhs = np.sum(lam * Sw)
        L = torch.tensor(lam, device="cuda")
        c.rk3_step_adjoint(Ud, dt, L)
        c.sync()
        rhs = np.sum(L.cpu().numpy() * w)
        assert abs(lhs - rhs) <= 1e-10 * abs(lhs), (lhs, rhs)
        c.close()


def test_sine_mode_gradient_against_tangent_linear_oracle():
    """dJ/da . da of the reduced sine-mode problem (N = 256, 200 steps, 8
    modes, checkpoints every 20): the adjoint gradient against the oracle's
    tangent-linear run along da, with dJ = 2 sum rho drho dx."""
    a = I.adjoint_modes(3, K=8)
    n, nsteps = 256, 200
    J, g, dt = A.sine_modes_gradient(a, n=n, nsteps=nsteps, every=20)
    rng = np.random.default_rng(17)
    for _ in range(3):
        da = rng.normal(size=a.size) * np.abs(a)
        U0, dx, x = I.adjoint_ic(a, n)
        # rho0 = 1 + sum a_k sin(2 pi k x), u0 = p0 = 1: drho0 = sum da_k sin(2 pi k x),
        # d(rho u)0 = drho0, dE0 = drho0 / 2
        s = np.sin(2 * np.pi * np.outer(x, np.arange(1, a.size + 1))) @ da
        dU0 = np.stack([s, s, 0.5 * s])
        UN, dUN = oracle.run_1d_tl(oracle.SYS_EULER1D, U0, dU0, dx, dt, nsteps, bc=(0, 0))
        assert float(np.sum(UN[0] ** 2) * dx) == pytest.approx(J, rel=1e-12)
        lhs = 2.0 * np.sum(UN[0] * dUN[0]) * dx
        rhs = float(np.dot(g, da))
        assert abs(lhs - rhs) <= 1e-10 * abs(lhs), (lhs, rhs)
