"""The per-field Lax-Friedrichs alpha on the GPU (t7_grid.alpha_mode =
T7_ALPHA_PER_FIELD, 1D Euler): alpha_k = max_i |lambda_k(U_i)| per
characteristic field and each field's split values (L_k F +- alpha_k L_k U)/2
in the face's Roe frame, against the oracle's alpha switch.  FP64 is
bit-identical to the oracle (RHS, masks, RK3 steps, whole runs); FP32 agrees
within the FP32 rounding bound.  The CFL step is the global alpha's.  Every
form outside 1D Euler with TENO7-ext in FP64 or FP32 refuses the mode."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1808_00037_gb300 import binding as B
from paper_1808_00037_gb300 import decomp
from paper_1808_00037_gb300 import inputs as I

pytestmark = pytest.mark.gpu

E1 = oracle.SYS_EULER1D
PF = B.T7_ALPHA_PER_FIELD


def _entropy_wave(n, u=0.4):
    x = (np.arange(n) + 0.5) / n
    rho = 1.0 + 0.3 * np.sin(2 * np.pi * x)
    return I.prim_to_cons_1d(rho, np.full(n, u), np.full(n, 1.0)), 1.0 / n


CASES = {
    "shu-osher": (lambda: I.shu_osher(1600), (1, 1)),
    "smooth-periodic": (lambda: I.random_euler_smooth(9, 301)[:2], (0, 0)),
    "sod": (lambda: I.riemann_tube(203, *I.SOD)[:2], (1, 1)),
    "entropy-wave": (lambda: _entropy_wave(256), (0, 0)),
}


def _ctx(n, dx, bc, prec):
    return B.Context(B.T7_EULER1D, n, dx, prec=prec, bc=tuple(bc) + (0, 0), gamma=1.4, alpha_mode=PF)


@pytest.mark.parametrize("name", list(CASES))
def test_rhs_f64_bitexact(name):
    (U, dx), bc = CASES[name][0](), CASES[name][1]
    with oracle.alpha_mode(oracle.ALPHA_PER_FIELD):
        ro, _, mo = oracle.rhs_1d(E1, U, dx, bc=bc, want_masks=True)
    c = _ctx(U.shape[1], dx, bc, B.T7_F64)
    rg, mg = c.euler_rhs(torch.tensor(U, device="cuda"), want_masks=True)
    c.sync()
    assert np.array_equal(rg.cpu().numpy(), ro)
    assert np.array_equal(mg.cpu().numpy(), mo)
    # and it is not the global-alpha RHS
    r0, _, _ = oracle.rhs_1d(E1, U, dx, bc=bc)
    assert not np.array_equal(ro, r0)
    c.close()


@pytest.mark.parametrize("name", ["shu-osher", "smooth-periodic", "sod"])
def test_rhs_f32_within_rounding_bound(name):
    (U, dx), bc = CASES[name][0](), CASES[name][1]
    with oracle.alpha_mode(oracle.ALPHA_PER_FIELD):
        ro, _, mo = oracle.rhs_1d(E1, U, dx, bc=bc, want_masks=True)
    c = _ctx(U.shape[1], dx, bc, B.T7_F32)
    rg, mg = c.euler_rhs(torch.tensor(U, dtype=torch.float32, device="cuda"), want_masks=True)
    c.sync()
    mg = mg.cpu().numpy()
    assert (mg == mo).mean() >= 0.999
    face_ok = np.all(mg == mo, axis=(0, 1))
    cell_ok = face_ok[:-1] & face_ok[1:]
    rho, u, pr = I.cons_to_prim_1d(U)
    fmax = np.max(np.abs(np.stack([U[1], U[1] * u + pr, u * (U[2] + pr)])))
    bound = 64 * 2.0**-24 * fmax / dx
    err = np.abs(rg.double().cpu().numpy() - ro)[:, cell_ok]
    assert np.max(err) <= bound, (np.max(err), bound)
    c.close()


def test_cfl_dt_is_the_global_alphas():
    U, dx = I.shu_osher(1600)
    dts = []
    for mode in (B.T7_ALPHA_GLOBAL, PF):
        c = B.Context(B.T7_EULER1D, 1600, dx, prec=B.T7_F64, bc=(1, 1, 0, 0), gamma=1.4, alpha_mode=mode)
        dts.append(c.cfl_dt(torch.tensor(U, device="cuda"), 0.5))
        c.close()
    with oracle.alpha_mode(oracle.ALPHA_PER_FIELD):
        do = oracle.cfl_dt_1d(E1, U, dx, 0.5)
    assert dts[0] == dts[1] == do


def test_rk3_step_f64_bitexact():
    U, dx = I.shu_osher(1600)
    dt = 0.5 * dx / oracle.alpha_1d(E1, U)
    with oracle.alpha_mode(oracle.ALPHA_PER_FIELD):
        Uo = oracle.rk3_step_1d(E1, U, dx, dt, bc=(1, 1))
    c = _ctx(1600, dx, (1, 1), B.T7_F64)
    Ug = torch.tensor(U, device="cuda")
    c.rk3_step(Ug, dt)
    c.sync()
    assert np.array_equal(Ug.cpu().numpy(), Uo)
    c.close()


@pytest.mark.parametrize("name,t_end,max_steps", [("shu-osher", 0.3, 1 << 30), ("smooth-periodic", math.inf, 40),
                                                 ("entropy-wave", 0.25, 1 << 30)])
def test_run_f64_bitexact(name, t_end, max_steps):
    (U, dx), bc = CASES[name][0](), CASES[name][1]
    with oracle.alpha_mode(oracle.ALPHA_PER_FIELD):
        Uo, so, to, _ = oracle.run_1d(E1, U, dx, t_end=t_end, cfl=0.5, bc=bc, max_steps=max_steps)
    c = _ctx(U.shape[1], dx, bc, B.T7_F64)
    Ug = torch.tensor(U, device="cuda")
    steps, t = c.run(Ug, 0.5, t_end=t_end, max_steps=max_steps)
    assert (steps, t) == (so, to)
    assert np.array_equal(Ug.cpu().numpy(), Uo)
    c.close()


def test_run_f32_follows_f64():
    """Shu-Osher N = 1600 to t = 1.8 in FP32 with per-field alphas: same step
    count as FP64, density within the shock-case FP32 tolerance."""
    U, dx = I.shu_osher(1600)
    out = {}
    for prec, dtype in ((B.T7_F64, torch.float64), (B.T7_F32, torch.float32)):
        c = _ctx(1600, dx, (1, 1), prec)
        Ug = torch.tensor(U, dtype=dtype, device="cuda")
        steps, t = c.run(Ug, 0.5, t_end=1.8)
        out[prec] = (steps, t, Ug.double().cpu().numpy())
        c.close()
    assert abs(out[B.T7_F32][0] - out[B.T7_F64][0]) <= 2
    r32, r64 = out[B.T7_F32][2][0], out[B.T7_F64][2][0]
    assert np.abs(r32 - r64).sum() / np.abs(r64).sum() < 2e-3
    rho, u, p = I.cons_to_prim_1d(out[B.T7_F32][2])
    assert np.all(rho > 0) and np.all(p > 0)


def test_other_forms_refuse_the_mode():
    U, dx = I.shu_osher(64)
    for kw in (dict(sys=B.T7_SCALAR_ADVECTION, prec=B.T7_F64), dict(sys=B.T7_BURGERS, prec=B.T7_F64),
               dict(sys=B.T7_EULER1D, prec=B.T7_MIXED), dict(sys=B.T7_EULER1D, prec=B.T7_F64, scheme=B.T7_TENO5)):
        sysid = kw.pop("sys")
        with pytest.raises(B.T7Error):
            B.Context(sysid, 64, dx, alpha_mode=PF, **kw)
    with pytest.raises(B.T7Error):
        B.Context(B.T7_EULER2D, 32, 0.1, ny=32, dy=0.1, alpha_mode=PF)
    with pytest.raises(B.T7Error):
        B.Context(B.T7_EULER1D, 64, dx, alpha_mode=2)
    c = _ctx(64, dx, (1, 1), B.T7_F64)
    Ug = torch.tensor(U, device="cuda")
    with pytest.raises(B.T7Error):
        c.run_host(torch.tensor(U).pin_memory(), 0.5, max_steps=1)
    with pytest.raises(B.T7Error):
        c.batch_run(Ug, np.array([0, 64], np.int64), np.array([dx]), 0.01, 0.5)
    with pytest.raises(B.T7Error):
        c.slab_alpha(decomp.padded(Ug), torch.zeros(1, dtype=torch.float64, device="cuda"))
    assert c.lib.t7_euler_rhs_adjoint(c.h, Ug.data_ptr(), Ug.data_ptr(), Ug.data_ptr()) == B.T7_EINVAL
    c.close()
