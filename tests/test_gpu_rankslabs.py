"""The rank-decomposed path on the GPU (paper_1808_00037_gb300.decomp.RankSlabs
over an NCCL process group with CUDA slab backends), as the bench's N-rank run
uses it.  Every run here has one GPU, so the group has one rank: its halos
come from the periodic wrap or the domain's boundary, and the all-reduce of
alpha goes through NCCL.  The run must equal the unsplit t7_run bit for bit
(steps, t and every value), in 1D (FP64, FP32) and 2D (FP32)."""
import math
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist

from paper_1808_00037_gb300 import binding as B
from paper_1808_00037_gb300 import decomp
from paper_1808_00037_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DTYPE = {B.T7_F64: torch.float64, B.T7_F32: torch.float32}


@pytest.fixture(scope="module")
def nccl_group():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("nccl", rank=0, world_size=1, device_id=torch.device("cuda", 0))
    yield
    dist.destroy_process_group()


@pytest.mark.parametrize("prec", [B.T7_F64, B.T7_F32])
@pytest.mark.parametrize("periodic", [False, True])
def test_rank_slab_1d_equals_unsplit(nccl_group, prec, periodic):
    if periodic:
        U, dx, _ = I.random_euler_smooth(9, 301)
        t_end, nsteps = math.inf, 30
    else:
        U, dx = I.shu_osher(1600)
        t_end, nsteps = 1.8, 40
    bc = (0, 0, 0, 0) if periodic else (1, 1, 0, 0)
    ctx = B.Context(B.T7_EULER1D, U.shape[1], dx, prec=prec, gamma=1.4)
    slab = decomp.Slab(decomp.CudaSlab(ctx), torch.tensor(U, dtype=DTYPE[prec], device="cuda"))
    steps, t = decomp.rk3_run_slabs(decomp.RankSlabs(slab, periodic), decomp.cfl_dt_1d(dx, 0.5), t_end=t_end,
                                    max_steps=nsteps)
    torch.cuda.synchronize()
    full = B.Context(B.T7_EULER1D, U.shape[1], dx, prec=prec, bc=bc, gamma=1.4)
    Ug = torch.tensor(U, dtype=DTYPE[prec], device="cuda")
    s_ref, t_ref = full.run(Ug, 0.5, t_end=t_end, max_steps=nsteps)
    assert (steps, t) == (s_ref, t_ref)
    assert torch.equal(slab.state(), Ug)
    ctx.close()
    full.close()


def test_rank_slab_2d_equals_unsplit(nccl_group):
    U, dx, dy, _ = I.quadrants_2d(3, 100, 90)
    _, ny, nx = U.shape
    ctx = B.Context(B.T7_EULER2D, nx, dx, ny=ny, dy=dy, prec=B.T7_F32, bc=(1, 1, 1, 1), gamma=1.4)
    slab = decomp.Slab(decomp.CudaSlab(ctx), torch.tensor(U, dtype=torch.float32, device="cuda"), nalpha=2)
    steps, t = decomp.rk3_run_slabs(decomp.RankSlabs(slab, False), decomp.cfl_dt_2d(dx, dy, 0.4), t_end=np.inf,
                                    max_steps=25)
    torch.cuda.synchronize()
    full = B.Context(B.T7_EULER2D, nx, dx, ny=ny, dy=dy, prec=B.T7_F32, bc=(1, 1, 1, 1), gamma=1.4)
    Ug = torch.tensor(U, dtype=torch.float32, device="cuda")
    s_ref, t_ref = full.run(Ug, 0.4, max_steps=25)
    assert (steps, t) == (s_ref, t_ref)
    assert torch.equal(slab.state(), Ug)
    ctx.close()
    full.close()
