"""The mixed-precision form (T7_MIXED): FP64 state, FP32 reconstruction, FP64
flux difference and RK combination.

* Its reconstruction is the FP32 kernel's: on the same (float-representable)
  state its stencil codes equal the FP32 path's exactly, and its RHS agrees
  with the FP32 path's within the FP32 bound (alpha is taken in FP64 here).
* Against the FP64 oracle: codes agree on >= 99.9% of entries and the RHS on
  agreeing faces is within 64 * 2^-24 * max|F| / dx (the FP32 bound).
* The face flux enters both neighbours as one FP64 value, so periodic domain
  sums are conserved to FP64 round-off (the FP32 state only to FP32's).
* Whole runs stay within the smooth-case tolerance of the FP64 oracle.
"""
import numpy as np
import pytest

import oracle
from paper_1808_00037_gb300 import binding as B
from paper_1808_00037_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SYSMAP = {oracle.SYS_ADVECTION: B.T7_SCALAR_ADVECTION, oracle.SYS_EULER1D: B.T7_EULER1D,
          oracle.SYS_BURGERS: B.T7_BURGERS}
CASES = [
    ("adv-sine", oracle.SYS_ADVECTION, lambda n: I.advection_sine(n)[:2], (0, 0), 1.0),
    ("burgers", oracle.SYS_BURGERS, lambda n: I.burgers_sine(n)[:2], (0, 0), 1.0),
    ("sod", oracle.SYS_EULER1D, lambda n: I.riemann_tube(n, *I.SOD)[:2], (1, 1), 1.0),
    ("shu-osher", oracle.SYS_EULER1D, lambda n: I.shu_osher(n), (1, 1), 1.0),
    ("euler-periodic", oracle.SYS_EULER1D, lambda n: I.random_euler_smooth(5, n)[:2], (0, 0), 1.0),
]


def ctx(sys, n, dx, prec, bc, a=1.0):
    return B.Context(SYSMAP[sys], n, dx, prec=prec, bc=(bc[0], bc[1], 0, 0), adv_speed=a)


def flux_max(sys, U, a):
    if sys == oracle.SYS_EULER1D:
        rho, u, pr = I.cons_to_prim_1d(U)
        return np.max(np.abs(np.stack([U[1], U[1] * u + pr, u * (U[2] + pr)])))
    return np.max(np.abs(U)) * max(abs(a), np.max(np.abs(U)))


@pytest.mark.parametrize("name,sys,gen,bc,a", CASES, ids=[c[0] for c in CASES])
def test_mixed_rhs_reconstruction_is_the_fp32_one(name, sys, gen, bc, a):
    n = 1600
    U, dx = gen(n)
    Uf = U.astype(np.float32).astype(np.float64)  # a state both forms hold exactly
    cm = ctx(sys, n, dx, B.T7_MIXED, bc, a)
    c32 = ctx(sys, n, dx, B.T7_F32, bc, a)
    rm, mm = cm.euler_rhs(torch.tensor(Uf, device="cuda"), want_masks=True)
    r32, m32 = c32.euler_rhs(torch.tensor(Uf, dtype=torch.float32, device="cuda"), want_masks=True)
    torch.cuda.synchronize()
    assert torch.equal(mm, m32)
    # alpha comes from the FP64 state in FP64 here and in FP32 on the FP32
    # path, so the split fluxes differ at FP32 rounding level: the FP32 bound
    bound = 64 * 2.0**-24 * flux_max(sys, Uf, a) / dx
    assert float((rm - r32.double()).abs().max()) <= bound


@pytest.mark.parametrize("name,sys,gen,bc,a", CASES, ids=[c[0] for c in CASES])
def test_mixed_rhs_against_oracle(name, sys, gen, bc, a):
    n = 1600
    U, dx = gen(n)
    ro, _, mo = oracle.rhs_1d(sys, U, dx, a=a, bc=bc, want_masks=True)
    c = ctx(sys, n, dx, B.T7_MIXED, bc, a)
    rg, mg = c.euler_rhs(torch.tensor(U, device="cuda"), want_masks=True)
    c.sync()
    mg = mg.cpu().numpy()
    assert (mg == mo).mean() >= 0.999
    face_ok = np.all(mg == mo, axis=(0, 1))
    cell_ok = face_ok[:-1] & face_ok[1:]
    err = np.abs(rg.cpu().numpy() - ro)[:, cell_ok]
    assert np.max(err) <= 64 * 2.0**-24 * flux_max(sys, U, a) / dx


NBIG = 1600 * 10486  # the tiled Shu-Osher workload: 16,777,600 cells


def test_mixed_conserves_domain_sums_to_fp64_roundoff():
    """At the benchmark size with periodic ends, three SSP-RK3 steps keep every
    domain sum to 1e-13 relative (the FP32 state holds them to ~1e-6)."""
    U, dx = I.shu_osher(1600, tiles=NBIG // 1600)
    c = ctx(oracle.SYS_EULER1D, U.shape[1], dx, B.T7_MIXED, (0, 0))
    Ug = torch.tensor(U, device="cuda")
    s0 = Ug.sum(dim=1)
    steps, _ = c.run(Ug, 0.5, max_steps=3)
    assert steps == 3
    s1 = Ug.sum(dim=1)
    assert torch.all(torch.abs(s1 - s0) <= 1e-13 * torch.abs(Ug).sum(dim=1)), (s0, s1)


def test_mixed_runs_against_oracle():
    """Smooth Euler to t = 0.2: within 1e-5 relative L1 of the FP64 oracle
    (the smooth-case tolerance); Shu-Osher N = 1600 to t = 1.8 within the
    FP32 path's bound; advection sine to t = 2 within 1e-5."""
    U, dx, _ = I.random_euler_smooth(7, 512)
    Uo, _, to, _ = oracle.run_1d(oracle.SYS_EULER1D, U, dx, t_end=0.2, cfl=0.5)
    c = ctx(oracle.SYS_EULER1D, 512, dx, B.T7_MIXED, (0, 0))
    Ug = torch.tensor(U, device="cuda")
    _, tg = c.run(Ug, 0.5, t_end=0.2)
    assert tg == to
    G = Ug.cpu().numpy()
    for k in range(3):
        assert np.abs(G[k] - Uo[k]).sum() / np.abs(Uo[k]).sum() < 1e-5
    U, dx = I.shu_osher(1600)
    Uo, _, _, _ = oracle.run_1d(oracle.SYS_EULER1D, U, dx, t_end=1.8, cfl=0.5, bc=(1, 1))
    c = ctx(oracle.SYS_EULER1D, 1600, dx, B.T7_MIXED, (1, 1))
    Ug = torch.tensor(U, device="cuda")
    c.run(Ug, 0.5, t_end=1.8)
    assert np.abs(Ug.cpu().numpy()[0] - Uo[0]).sum() / np.abs(Uo[0]).sum() < 2e-3
    U, dx, _ = I.advection_sine(200)
    Uo, _, _, _ = oracle.run_1d(oracle.SYS_ADVECTION, U, dx, t_end=2.0, cfl=0.2)
    c = ctx(oracle.SYS_ADVECTION, 200, dx, B.T7_MIXED, (0, 0))
    Ug = torch.tensor(U, device="cuda")
    c.run(Ug, 0.2, t_end=2.0)
    assert np.abs(Ug.cpu().numpy()[0] - Uo[0]).sum() / np.abs(Uo[0]).sum() < 1e-5


def test_mixed_host_run_and_refusals():
    U, dx = I.shu_osher(1600)
    c = ctx(oracle.SYS_EULER1D, 1600, dx, B.T7_MIXED, (1, 1))
    Ud = torch.tensor(U, device="cuda")
    sd, td = c.run(Ud, 0.5, max_steps=11)
    Uh = np.ascontiguousarray(U)
    sh, th = c.run_host(Uh, 0.5, max_steps=11)
    assert (sd, td) == (sh, th)
    assert np.array_equal(Ud.cpu().numpy(), Uh)
    with pytest.raises(B.T7Error):
        c.euler_rhs_adjoint(Ud, Ud.clone())
    with pytest.raises(B.T7Error):
        c.batch_run(Ud, [0, 1600], [dx], t_end=0.01, cfl=0.5)
    with pytest.raises(B.T7Error):
        c.teno7_reconstruct(torch.zeros(72, dtype=torch.float64, device="cuda"), 1, 1e-6)
