"""GPU parity of the TENO5 baseline (the fifth-order TENO scheme of Sec. 2,
Table co1) against the oracle run with its TENO5 switch.

FP64 is compared bit for bit (right-hand sides, the three-bit codes the faces
select with, RK steps and whole runs); FP32 against the FP64 oracle with the
same bounds as the TENO7-ext path.  Entry points that only run TENO7-ext
refuse a TENO5 context.
"""
import numpy as np
import pytest

import oracle
from oracle import riemann
from paper_1808_00037_gb300 import binding as B
from paper_1808_00037_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SYSMAP = {oracle.SYS_ADVECTION: B.T7_SCALAR_ADVECTION, oracle.SYS_EULER1D: B.T7_EULER1D,
          oracle.SYS_BURGERS: B.T7_BURGERS}

CASES = [
    ("adv-sine", oracle.SYS_ADVECTION, lambda n: I.advection_sine(n)[:2], (0, 0), 1.0),
    ("adv-neg", oracle.SYS_ADVECTION, lambda n: I.random_smooth_1d(3, n)[:2], (0, 0), -0.7),
    ("burgers", oracle.SYS_BURGERS, lambda n: I.burgers_sine(n)[:2], (0, 0), 1.0),
    ("sod", oracle.SYS_EULER1D, lambda n: I.riemann_tube(n, *I.SOD)[:2], (1, 1), 1.0),
    ("lax", oracle.SYS_EULER1D, lambda n: I.riemann_tube(n, *I.LAX)[:2], (1, 1), 1.0),
    ("shu-osher", oracle.SYS_EULER1D, lambda n: I.shu_osher(n), (1, 1), 1.0),
    ("euler-periodic", oracle.SYS_EULER1D, lambda n: I.random_euler_smooth(5, n)[:2], (0, 0), 1.0),
]


def ctx(sys, n, dx, prec=B.T7_F64, bc=(0, 0), a=1.0):
    return B.Context(SYSMAP[sys], n, dx, prec=prec, bc=(bc[0], bc[1], 0, 0), adv_speed=a, scheme=B.T7_TENO5)


def dev(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def host(t):
    return t.double().cpu().numpy()


def rel_l1(a, b):
    return np.abs(a - b).sum() / np.abs(b).sum()


@pytest.fixture(autouse=True)
def teno5_oracle():
    with oracle.scheme(oracle.SCHEME_TENO5):
        yield


@pytest.mark.parametrize("name,sys,gen,bc,a", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("n", [3, 200, 759, 1600])
def test_teno5_rhs_f64_bitexact(name, sys, gen, bc, a, n):
    U, dx = gen(n)
    ro, _, mo = oracle.rhs_1d(sys, U, dx, a=a, bc=bc, want_masks=True)
    assert mo.max() <= 7
    c = ctx(sys, n, dx, bc=bc, a=a)
    rg, mg = c.euler_rhs(dev(U), want_masks=True)
    c.sync()
    assert np.array_equal(mg.cpu().numpy(), mo)
    assert np.array_equal(host(rg), ro)


@pytest.mark.parametrize("name,sys,gen,bc,a", CASES, ids=[c[0] for c in CASES])
def test_teno5_rk3_step_f64_bitexact(name, sys, gen, bc, a):
    n = 1600
    U, dx = gen(n)
    dt = 0.5 * oracle.cfl_dt_1d(sys, U, dx, 1.0, a=a)
    Uo = oracle.rk3_step_1d(sys, U, dx, dt, a=a, bc=bc)
    c = ctx(sys, n, dx, bc=bc, a=a)
    Ug = dev(U)
    c.rk3_step(Ug, dt)
    c.sync()
    assert np.array_equal(host(Ug), Uo)


def test_teno5_shu_osher_run_f64_bitexact():
    """Shu-Osher, N = 1600, CFL 0.5 to t = 1.8 with TENO5: identical to the oracle."""
    U, dx = I.shu_osher(1600)
    Uo, so, to, _ = oracle.run_1d(oracle.SYS_EULER1D, U, dx, t_end=1.8, cfl=0.5, bc=(1, 1))
    c = ctx(oracle.SYS_EULER1D, 1600, dx, bc=(1, 1))
    Ug = dev(U)
    sg, tg = c.run(Ug, 0.5, t_end=1.8)
    assert (sg, tg) == (so, to)
    assert np.array_equal(host(Ug), Uo)


def test_teno5_sod_against_exact_riemann():
    U, dx, x = I.riemann_tube(200, *I.SOD)
    rho, _, _ = riemann.sample(*I.SOD, (x - 0.5) / 0.2)
    for prec, dtype in ((B.T7_F64, torch.float64), (B.T7_F32, torch.float32)):
        c = ctx(oracle.SYS_EULER1D, 200, dx, bc=(1, 1), prec=prec)
        Ug = dev(U, dtype)
        c.run(Ug, 0.6, t_end=0.2)
        assert np.mean(np.abs(host(Ug)[0] - rho)) < 6e-3


def window_variation(sys, U, bc, a):
    """Relative variation (max - min) / max|w| of the five characteristic
    values each face's smoothness measure reads, per [split][field][face]
    (faces j+1/2, j = -1 .. n-1; '+' window cells j-2 .. j+2, '-' window
    cells j+3 .. j-1), from the split fluxes G = (F +- alpha U) / 2 projected
    with the oracle's Roe frame of the face.  Also returns max|w| per entry."""
    m, n = U.shape
    P = np.pad(U, ((0, 0), (4, 4)), mode="wrap" if bc[0] == 0 else "edge")
    alpha = oracle.alpha_1d(sys, U, a=a)
    if sys == oracle.SYS_ADVECTION:
        F = a * P
    elif sys == oracle.SYS_BURGERS:
        F = 0.5 * P * P
    else:
        rho, u, pr = I.cons_to_prim_1d(P)
        F = np.stack([P[1], P[1] * u + pr, u * (P[2] + pr)])
    G = (0.5 * (F + alpha * P), 0.5 * (F - alpha * P))
    var = np.zeros((2, m, n + 1))
    qmax = np.zeros((2, m, n + 1))
    for f in range(n + 1):
        c = f + 3  # padded index of cell j = f - 1
        L = oracle.frame_1d(P[:, c], P[:, c + 1])[0] if m == 3 else np.eye(1)
        for sgn, cells in ((0, range(c - 2, c + 3)), (1, range(c - 1, c + 4))):
            w = L @ G[sgn][:, list(cells)]
            top = np.max(np.abs(w), axis=1)
            var[sgn, :, f] = np.where(top > 0, (w.max(axis=1) - w.min(axis=1)) / np.where(top > 0, top, 1), 0)
            qmax[sgn, :, f] = top
    return var, qmax


@pytest.mark.parametrize("name,sys,gen,bc,a", CASES, ids=[c[0] for c in CASES])
def test_teno5_rhs_f32_masks_and_values(name, sys, gen, bc, a):
    """FP32 against the FP64 oracle.  Where a sub-stencil of a face's
    characteristic window is constant in exact arithmetic (a constant state, a
    field whose projection does not see the varying variable -- the u - c
    field where u = 0 and p is uniform -- or the flat side of a jump) its beta
    is pure round-off, and against TENO5's epsilon of 1e-40 that round-off
    decides the FP64 cutoff (the defect the paper's epsilon = dx^3 removes);
    the FP32 kernel floors epsilon at its round-off level 2^-24 Q^2 / 12.  So:
    * codes agree on >= 99% of the entries whose oracle code is the same with
      epsilon = 1e-40 and with epsilon at the largest FP32 floor of the
      state (the entries the floor cannot move);
    * the RHS is within 64 * 2^-24 * max|F| / dx on every cell whose two faces
      agree on each entry or have a window flat to 1e-9 (any Table co1 row
      returns a constant window's value), and that is >= 90% of the cells."""
    n = 1600
    U, dx = gen(n)
    ro, _, mo = oracle.rhs_1d(sys, U, dx, a=a, bc=bc, want_masks=True)
    c = ctx(sys, n, dx, bc=bc, a=a, prec=B.T7_F32)
    rg, mg = c.euler_rhs(dev(U, torch.float32), want_masks=True)
    c.sync()
    mg = mg.cpu().numpy()
    var, qmax = window_variation(sys, U, bc, a)
    eps_hi = 2.0**-24 / 12 * float(np.max(qmax)) ** 2
    _, _, mh = oracle.rhs_1d(sys, U, dx, a=a, bc=bc, want_masks=True, eps=eps_hi)
    firm = mo == mh
    assert (mg == mo)[firm].mean() >= 0.99, (mg == mo)[firm].mean()
    face_ok = np.all((mg == mo) | (var < 1e-9), axis=(0, 1))
    cell_ok = face_ok[:-1] & face_ok[1:]
    assert cell_ok.mean() >= 0.9, cell_ok.mean()
    err = np.abs(host(rg) - ro)[:, cell_ok]
    if sys == oracle.SYS_EULER1D:
        rho, u, pr = I.cons_to_prim_1d(U)
        fmax = np.max(np.abs(np.stack([U[1], U[1] * u + pr, u * (U[2] + pr)])))
    else:
        fmax = np.max(np.abs(U)) * max(abs(a), np.max(np.abs(U)))
    assert np.max(err) <= 64 * 2.0**-24 * fmax / dx


def test_teno5_f32_smooth_run_tolerance():
    U, dx, x = I.advection_sine(200)
    Uo, _, _, _ = oracle.run_1d(oracle.SYS_ADVECTION, U, dx, t_end=2.0, cfl=0.2)
    c = ctx(oracle.SYS_ADVECTION, 200, dx, prec=B.T7_F32)
    Ug = dev(U, torch.float32)
    c.run(Ug, 0.2, t_end=2.0)
    assert rel_l1(host(Ug)[0], Uo[0]) < 1e-5


NBIG = 1600 * 10486  # the tiled Shu-Osher workload: 16,777,600 cells


def test_teno5_full_size_rhs_sampled_f64():
    """At the benchmark's size, TENO5 RHS on sampled cells against the oracle
    on windows around them (cell i depends on cells i-3 .. i+3 and alpha)."""
    U, dx = I.shu_osher(1600, tiles=NBIG // 1600)
    n = U.shape[1]
    alpha = oracle.alpha_1d(oracle.SYS_EULER1D, U)
    c = ctx(oracle.SYS_EULER1D, n, dx, bc=(1, 1))
    rg, mg = c.euler_rhs(dev(U), want_masks=True)
    c.sync()
    rng = np.random.default_rng(19)
    idx = np.concatenate([[0, 1, 2, 28, 29, n - 1, n - 2, n - 5], rng.integers(0, n, 200)])
    W = 12
    for i in idx:
        lo, hi = max(0, i - W), min(n, i + W + 1)
        ro, _, mo = oracle.rhs_1d(oracle.SYS_EULER1D, U[:, lo:hi], dx, bc=(1, 1), alpha=alpha, want_masks=True)
        k = i - lo
        if (lo > 0 and k < 6) or (hi < n and (hi - lo) - k < 7):
            continue
        assert np.array_equal(host(rg[:, i:i + 1])[:, 0], ro[:, k]), i
        assert np.array_equal(mg[:, :, i].cpu().numpy(), mo[:, :, k]), i


def test_teno5_refused_where_only_teno7ext_runs():
    U, dx = I.shu_osher(64)
    c = ctx(oracle.SYS_EULER1D, 64, dx, bc=(1, 1))
    Ug = dev(U)
    with pytest.raises(B.T7Error) as ei:
        c.euler_rhs_adjoint(Ug, Ug.clone())
    assert ei.value.status == B.T7_EINVAL
    with pytest.raises(B.T7Error):
        c.batch_run(Ug, [0, 64], [dx], t_end=0.01, cfl=0.5)
    with pytest.raises(B.T7Error):
        c.teno7_reconstruct(dev(np.zeros(72)), 1, 1e-6)
    with pytest.raises(B.T7Error):
        c.rk3_step_static(Ug, 1e-4)
    with pytest.raises(B.T7Error):
        B.Context(B.T7_EULER2D, 16, 0.1, ny=16, dy=0.1, scheme=B.T7_TENO5)
    # the context still runs its own scheme afterwards
    steps, _ = c.run(Ug, 0.5, max_steps=2)
    assert steps == 2
