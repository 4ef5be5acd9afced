"""The decomposed 1D path on the GPU: slabs of one domain, each with its own
context on its own CUDA stream, padded by 4 halo cells per side that are
filled by device-local copies, advanced by t7_slab_stage with the alpha of
every stage all-reduced (a max over the slabs) on the device
(paper_1808_00037_gb300.decomp.LocalSlabs).  The stencil reach of Eq. app sets
the halo, and the global Lax-Friedrichs alpha of Sec. "One dimensional Euler
equations" is one value for the whole domain; with both exchanged, every
slab computes exactly what the unsplit kernels compute, so the results must
be bit-identical to the unsplit run (FP64, FP32, mixed) and, in FP64, to the
oracle."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1808_00037_gb300 import binding as B
from paper_1808_00037_gb300 import decomp
from paper_1808_00037_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DTYPE = {B.T7_F64: torch.float64, B.T7_F32: torch.float32, B.T7_MIXED: torch.float64}


def _case(name):
    if name == "shu-osher":
        U, dx = I.shu_osher(1600)
        return B.T7_EULER1D, U, dx, False, 1.8, 40
    if name == "smooth-periodic":
        U, dx, _ = I.random_euler_smooth(9, 301)
        return B.T7_EULER1D, U, dx, True, math.inf, 30
    U, dx, _ = I.burgers_sine(160)
    return B.T7_BURGERS, U, dx, True, 1.5 / math.pi, 200


def _slabs(sysid, U, dx, prec, nslabs, periodic):
    slabs = []
    for r in range(nslabs):
        lo, hi = decomp.partition(U.shape[1], nslabs, r)
        st = torch.cuda.Stream()
        ctx = B.Context(sysid, hi - lo, dx, prec=prec, gamma=1.4, stream=st)
        Ul = torch.tensor(U[:, lo:hi], dtype=DTYPE[prec], device="cuda")
        slabs.append(decomp.Slab(decomp.CudaSlab(ctx), Ul))
    torch.cuda.synchronize()
    return decomp.LocalSlabs(slabs, periodic)


@pytest.mark.parametrize("prec", [B.T7_F64, B.T7_F32, B.T7_MIXED])
@pytest.mark.parametrize("name", ["shu-osher", "smooth-periodic", "burgers"])
def test_slab_rhs_equals_unsplit_rhs(prec, name):
    """L(U) and the Delta masks of each padded slab, with halos from the
    neighbouring slabs (or the domain's boundary condition) and the global
    alpha, equal the unsplit t7_euler_rhs on the slab's cells bit for bit."""
    sysid, U, dx, periodic, _, _ = _case(name)
    bc = (0, 0, 0, 0) if periodic else (1, 1, 0, 0)
    full = B.Context(sysid, U.shape[1], dx, prec=prec, bc=bc, gamma=1.4)
    Ug = torch.tensor(U, dtype=DTYPE[prec], device="cuda")
    L, masks = full.euler_rhs(Ug, want_masks=True)
    comm = _slabs(sysid, U, dx, prec, 3, periodic)
    comm.fill_halos(0)
    for s in comm.slabs:
        with torch.cuda.stream(s.stream):
            s.backend.alpha(s.P[0], s.a[0])
    g = torch.zeros(1, dtype=torch.float64, device="cuda")
    comm.allreduce_max(0, g)
    lo = 0
    for s in comm.slabs:
        with torch.cuda.stream(s.stream):
            Ls, ms = s.backend.ctx.slab_rhs(s.P[0], g, want_masks=True)
        s.stream.synchronize()
        n = Ls.shape[1]
        assert torch.equal(Ls, L[:, lo:lo + n]), (name, lo)
        # faces lo-1/2 .. lo+n-1/2 of the domain are the slab's faces -1 .. n-1
        assert torch.equal(ms, masks[:, :, lo:lo + n + 1]), (name, lo)
        lo += n
        s.backend.ctx.close()
    full.close()


@pytest.mark.parametrize("nslabs", [2, 3])
@pytest.mark.parametrize("prec", [B.T7_F64, B.T7_F32, B.T7_MIXED])
@pytest.mark.parametrize("name", ["shu-osher", "smooth-periodic", "burgers"])
def test_slabs_on_streams_bit_identical(nslabs, prec, name):
    """A run split into 2 or 3 slabs on separate streams equals the unsplit
    t7_run (steps, t and every value), and in FP64 the oracle's run."""
    sysid, U, dx, periodic, t_end, max_steps = _case(name)
    bc = (0, 0, 0, 0) if periodic else (1, 1, 0, 0)
    comm = _slabs(sysid, U, dx, prec, nslabs, periodic)
    steps, t = decomp.rk3_run_slabs(comm, decomp.cfl_dt_1d(dx, 0.5), t_end=t_end, max_steps=max_steps)
    torch.cuda.synchronize()
    got = torch.cat([s.state() for s in comm.slabs], dim=1)
    full = B.Context(sysid, U.shape[1], dx, prec=prec, bc=bc, gamma=1.4)
    Ug = torch.tensor(U, dtype=DTYPE[prec], device="cuda")
    s_ref, t_ref = full.run(Ug, 0.5, t_end=t_end, max_steps=max_steps)
    assert (steps, t) == (s_ref, t_ref)
    assert torch.equal(got, Ug)
    if prec == B.T7_F64:
        osys = {B.T7_EULER1D: oracle.SYS_EULER1D, B.T7_BURGERS: oracle.SYS_BURGERS}[sysid]
        Uo, so, to, _ = oracle.run_1d(osys, U, dx, t_end=t_end, cfl=0.5, bc=bc[:2], max_steps=max_steps)
        assert (so, to) == (steps, t)
        assert np.array_equal(got.cpu().numpy(), Uo)
    for s in comm.slabs:
        s.backend.ctx.close()
    full.close()


def test_slab_calls_reject_bad_arguments():
    """Aliased stage input and output, a bad stage index, an unpadded array
    and a non-float64 alpha are refused before any launch."""
    U, dx = I.shu_osher(64)
    ctx = B.Context(B.T7_EULER1D, 64, dx, prec=B.T7_F64, gamma=1.4)
    P = decomp.padded(torch.tensor(U, device="cuda"))
    Q = torch.zeros_like(P)
    a = torch.ones(1, dtype=torch.float64, device="cuda")
    lib = ctx.lib
    assert lib.t7_slab_stage(ctx.h, 0, P.data_ptr(), None, P.data_ptr(), a.data_ptr(), 1e-3, None) == B.T7_EINVAL
    assert lib.t7_slab_stage(ctx.h, 3, P.data_ptr(), P.data_ptr(), Q.data_ptr(), a.data_ptr(), 1e-3,
                             None) == B.T7_EINVAL
    assert lib.t7_slab_stage(ctx.h, 1, P.data_ptr(), None, Q.data_ptr(), a.data_ptr(), 1e-3, None) == B.T7_EINVAL
    assert lib.t7_slab_stage(ctx.h, 0, P.data_ptr(), None, Q.data_ptr(), None, 1e-3, None) == B.T7_EINVAL
    with pytest.raises(ValueError):
        ctx.slab_stage(0, torch.tensor(U, device="cuda"), None, Q, a, 1e-3)
    P[:, :4] = P[:, 4:5]  # zero-gradient halos, so that the accepted call below sees a valid state
    P[:, -4:] = P[:, -5:-4]
    with pytest.raises(ValueError):
        ctx.slab_stage(0, P, None, Q, a.float(), 1e-3)
    ctx.slab_stage(0, P, None, Q, a, 1e-3)
    ctx.sync()
    ctx.close()
