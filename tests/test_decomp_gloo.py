"""Multi-rank path on CPU: the slab decomposition (4-cell halo exchange and
all-reduce(max) of alpha per RK stage, all-reduce of the CFL step) with gloo
ranks, each rank computing its padded slab's RHS with the oracle.  The
gathered result must be bit-identical to the unsplit oracle run, which pins
the halo width, the boundary handling at the domain ends and the
synchronisation of alpha and dt."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_1808_00037_gb300 import decomp
from paper_1808_00037_gb300 import inputs as I


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _case(name):
    if name == "sod":
        U, dx, _ = I.riemann_tube(203, *I.SOD)
        return U, dx, False, 0.05, 1 << 30
    if name == "shu-osher":
        U, dx = I.shu_osher(400)
        return U, dx, False, 0.3, 1 << 30
    U, dx, _ = I.random_euler_smooth(9, 257)
    return U, dx, True, np.inf, 25


def _worker(rank, world, port, name):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        U, dx, periodic, t_end, max_steps = _case(name)
        bc = (0, 0) if periodic else (1, 1)
        lo, hi = decomp.partition(U.shape[1], world, rank)

        def rhs(P, alpha):
            return oracle.rhs_1d(oracle.SYS_EULER1D, P, dx, bc=(1, 1), alpha=alpha)[0]

        def alpha_local(X):
            return oracle.alpha_1d(oracle.SYS_EULER1D, X)

        Ul, steps, t = decomp.rk3_run(U[:, lo:hi], rhs, alpha_local, dx=dx, cfl=0.5, t_end=t_end,
                                      max_steps=max_steps, periodic=periodic)
        parts = [None] * world
        dist.all_gather_object(parts, (lo, hi, Ul, steps, t))
        if rank == 0:
            Uo, so, to, st = oracle.run_1d(oracle.SYS_EULER1D, U, dx, t_end=t_end, cfl=0.5, bc=bc,
                                           max_steps=max_steps)
            full = np.concatenate([p[2] for p in sorted(parts, key=lambda p: p[0])], axis=1)
            assert all(p[3] == so and p[4] == to for p in parts), (so, to, [(p[3], p[4]) for p in parts])
            assert np.array_equal(full, Uo)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("name", ["sod", "shu-osher", "smooth-periodic"])
def test_slab_decomposition_bit_identical(world, name):
    mp.spawn(_worker, args=(world, _free_port(), name), nprocs=world, join=True)


def test_partition_covers_domain():
    for n in (4, 7, 100, 1601):
        for world in (1, 2, 3, 8):
            if n < 4 * world:
                continue
            ranges = [decomp.partition(n, world, r) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
            sizes = [h - l for l, h in ranges]
            assert max(sizes) - min(sizes) <= 1
