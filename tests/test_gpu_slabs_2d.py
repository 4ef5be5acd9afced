"""The decomposed 2D path on the GPU: a 2D Euler domain cut along y into
slabs, each with its own context on its own CUDA stream and padded by 4 halo
rows per side that device-local copies fill, advanced by t7_slab_stage with
both wave speeds (alpha_x, alpha_y) of every stage all-reduced (a max over
the slabs) on the device (paper_1808_00037_gb300.decomp.LocalSlabs).  The
scheme is applied dimension by dimension (Remark 3's frame per direction), so
the y stencils reach 4 rows per side (Eq. app, Eq. vec) and the x direction
stays whole in every slab; with the halos and the global alphas exchanged,
every slab computes exactly what the unsplit kernels compute.  So the
results must be bit-identical to the unsplit run (FP64, FP32, mixed) and, in
FP64, to the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1808_00037_gb300 import binding as B
from paper_1808_00037_gb300 import decomp
from paper_1808_00037_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DTYPE = {B.T7_F64: torch.float64, B.T7_F32: torch.float32, B.T7_MIXED: torch.float64}
CFL = 0.4


def _case(name):
    """(U[4, ny, nx], dx, dy, periodic, steps).  Sizes ragged against the
    kernels' 29-row, 32-column and 29-cell tiles; every slab spans more than
    one 29-row block."""
    if name == "quadrants":
        U, dx, dy, _ = I.quadrants_2d(3, 100, 90)
        return U, dx, dy, False, 30
    U, dx, dy = I.random_smooth_2d(4, 70, 97)
    return U, dx, dy, True, 20


def _bc(periodic):
    return (0, 0, 0, 0) if periodic else (1, 1, 1, 1)


def _slabs(U, dx, dy, prec, nslabs, periodic):
    _, ny, nx = U.shape
    slabs = []
    for r in range(nslabs):
        lo, hi = decomp.partition(ny, nslabs, r)
        st = torch.cuda.Stream()
        # bc[0..1] act in x; the y ends come from the halos
        ctx = B.Context(B.T7_EULER2D, nx, dx, ny=hi - lo, dy=dy, prec=prec, bc=_bc(periodic), gamma=1.4,
                        stream=st)
        Ul = torch.tensor(U[:, lo:hi], dtype=DTYPE[prec], device="cuda")
        slabs.append(decomp.Slab(decomp.CudaSlab(ctx), Ul, nalpha=2))
    torch.cuda.synchronize()
    return decomp.LocalSlabs(slabs, periodic)


@pytest.mark.parametrize("prec", [B.T7_F64, B.T7_F32, B.T7_MIXED])
@pytest.mark.parametrize("name", ["quadrants", "smooth-periodic"])
def test_slab2d_rhs_equals_unsplit_rhs(prec, name):
    """L(U) and both sweeps' Delta masks of each padded slab, with halo rows
    from the neighbouring slabs (or the domain's y boundary condition) and the
    global alphas, equal the unsplit t7_euler_rhs on the slab's rows bit for
    bit; the slabs' alphas all-reduce to the unsplit run's."""
    U, dx, dy, periodic, _ = _case(name)
    _, ny, nx = U.shape
    full = B.Context(B.T7_EULER2D, nx, dx, ny=ny, dy=dy, prec=prec, bc=_bc(periodic), gamma=1.4)
    Ug = torch.tensor(U, dtype=DTYPE[prec], device="cuda")
    L, (xm, ym) = full.euler_rhs(Ug, want_masks=True)
    comm = _slabs(U, dx, dy, prec, 3, periodic)
    comm.fill_halos(0)
    for s in comm.slabs:
        with torch.cuda.stream(s.stream):
            s.backend.alpha(s.P[0], s.a[0])
    g = torch.zeros(2, dtype=torch.float64, device="cuda")
    comm.allreduce_max(0, g)
    if prec == B.T7_F32:
        # from the FP32 state in FP32 arithmetic
        sx, sy = _wave_speeds(U.astype(np.float32).astype(np.float64))
        assert np.allclose(g.cpu().numpy(), [sx, sy], rtol=1e-6, atol=0)
    else:
        # an FP64 state: the oracle's alphas exactly
        _, (ax, ay), _ = oracle.rhs_2d(U, dx, dy, bc=_bc(periodic))
        assert g.cpu().tolist() == [ax, ay]
    lo = 0
    for s in comm.slabs:
        with torch.cuda.stream(s.stream):
            Ls, (sxm, sym) = s.backend.ctx.slab_rhs(s.P[0], g, want_masks=True)
        s.stream.synchronize()
        n = Ls.shape[1]
        assert torch.equal(Ls, L[:, lo:lo + n]), (name, lo)
        assert torch.equal(sxm, xm[:, :, lo:lo + n]), (name, lo)
        # y faces lo-1/2 .. lo+n-1/2 of the domain are the slab's faces -1 .. n-1
        assert torch.equal(sym, ym[:, :, :, lo:lo + n + 1]), (name, lo)
        lo += n
        s.backend.ctx.close()
    full.close()


def _wave_speeds(U):
    """max(|u| + c), max(|v| + c) of a 2D state, in FP64 (gamma = 1.4)."""
    rho, mu, mv, E = U
    u, v = mu / rho, mv / rho
    p = 0.4 * (E - 0.5 * (mu * u + mv * v))
    c = np.sqrt(1.4 * p / rho)
    return float(np.max(np.abs(u) + c)), float(np.max(np.abs(v) + c))


@pytest.mark.parametrize("nslabs", [2, 3])
@pytest.mark.parametrize("prec", [B.T7_F64, B.T7_F32, B.T7_MIXED])
@pytest.mark.parametrize("name", ["quadrants", "smooth-periodic"])
def test_slabs2d_on_streams_bit_identical(nslabs, prec, name):
    """A 2D run split along y into 2 or 3 slabs on separate streams equals the
    unsplit t7_run (steps, t and every value), and in FP64 the oracle's run."""
    U, dx, dy, periodic, nsteps = _case(name)
    _, ny, nx = U.shape
    comm = _slabs(U, dx, dy, prec, nslabs, periodic)
    steps, t = decomp.rk3_run_slabs(comm, decomp.cfl_dt_2d(dx, dy, CFL), t_end=np.inf, max_steps=nsteps)
    torch.cuda.synchronize()
    got = torch.cat([s.state() for s in comm.slabs], dim=1)
    full = B.Context(B.T7_EULER2D, nx, dx, ny=ny, dy=dy, prec=prec, bc=_bc(periodic), gamma=1.4)
    Ug = torch.tensor(U, dtype=DTYPE[prec], device="cuda")
    s_ref, t_ref = full.run(Ug, CFL, max_steps=nsteps)
    assert (steps, t) == (s_ref, t_ref)
    assert torch.equal(got, Ug)
    if prec == B.T7_F64:
        Uo, so, to, _ = oracle.run_2d(U, dx, dy, cfl=CFL, max_steps=nsteps, bc=_bc(periodic))
        assert (so, to) == (steps, t)
        assert np.array_equal(got.cpu().numpy(), Uo)
    for s in comm.slabs:
        s.backend.ctx.close()
    full.close()


def test_slab2d_calls_reject_bad_arguments():
    """An unpadded array, a one-element alpha and an aliased stage input and
    output are refused before any launch; a well-formed call is accepted."""
    U, dx, dy, _ = I.quadrants_2d(3, 40, 36)
    ctx = B.Context(B.T7_EULER2D, 40, dx, ny=36, dy=dy, prec=B.T7_F64, bc=(1, 1, 1, 1))
    P = decomp.padded(torch.tensor(U, device="cuda"))
    P[:, :4] = P[:, 4:5]  # zero-gradient halo rows: a valid state for the accepted call
    P[:, -4:] = P[:, -5:-4]
    Q = torch.zeros_like(P)
    a = torch.ones(2, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        ctx.slab_stage(0, torch.tensor(U, device="cuda"), None, Q, a, 1e-4)
    with pytest.raises(ValueError):
        ctx.slab_stage(0, P, None, Q, a[:1], 1e-4)
    assert ctx.lib.t7_slab_stage(ctx.h, 0, P.data_ptr(), None, P.data_ptr(), a.data_ptr(), 1e-4,
                                 None) == B.T7_EINVAL
    ao = torch.zeros(2, dtype=torch.float64, device="cuda")
    ctx.slab_stage(0, P, None, Q, a, 1e-4, ao)
    ctx.sync()
    assert bool((ao > 0).all())
    ctx.close()
