"""Multi-rank path on CPU: the slab decomposition (4-cell halo exchange and
all-reduce(max) of alpha per RK stage, all-reduce of the CFL step) with gloo
ranks, each rank computing its padded slab's RHS with the oracle.  The
gathered result must be bit-identical to the unsplit oracle run, which pins
the halo width, the boundary handling at the domain ends and the
synchronisation of alpha and dt."""
import socket

import numpy as np
import pytest
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


def _case2d(name):
    if name == "quadrants":
        U, dx, dy, _ = I.quadrants_2d(3, 26, 30)
        return U, dx, dy, False, 6
    U, dx, dy = I.random_smooth_2d(4, 24, 28)
    return U, dx, dy, True, 6


def _worker2d(rank, world, port, name):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        U, dx, dy, periodic, nsteps = _case2d(name)
        bcx = (0, 0) if periodic else (1, 1)
        lo, hi = decomp.partition(U.shape[1], world, rank)

        def rhs(P, alpha):
            return oracle.rhs_2d(P, dx, dy, bc=(bcx[0], bcx[1], 1, 1), alpha=alpha)[0]

        Ul, steps, t = decomp.rk3_run_2d(U[:, lo:hi], rhs, oracle.alpha_2d, dx=dx, dy=dy, cfl=0.4,
                                         t_end=np.inf, max_steps=nsteps, periodic_y=periodic)
        sums = decomp.global_sums(Ul)
        parts = [None] * world
        dist.all_gather_object(parts, (lo, Ul, steps, t))
        if rank == 0:
            bc = (0, 0, 0, 0) if periodic else (1, 1, 1, 1)
            Uo, so, to, st = oracle.run_2d(U, dx, dy, cfl=0.4, max_steps=nsteps, bc=bc)
            full = np.concatenate([p[1] for p in sorted(parts, key=lambda p: p[0])], axis=1)
            assert all(p[2] == so and p[3] == to for p in parts)
            assert np.array_equal(full, Uo)
            assert np.allclose(sums, Uo.reshape(4, -1).sum(axis=1), rtol=1e-14, atol=0)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("name", ["quadrants", "smooth-periodic"])
def test_2d_slab_decomposition_bit_identical(world, name):
    """2D split along y: 4 halo rows per side, both alphas all-reduced at every
    stage, the CFL step cfl / (ax/dx + ay/dy); gathered result bit-identical to
    the unsplit oracle run; FP64 all-reduced domain sums equal the full sums."""
    mp.spawn(_worker2d, args=(world, _free_port(), name), nprocs=world, join=True)


def _worker_tubes(rank, world, port):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        U, off, dx, _ = I.riemann_tube_batch(3, 12, 24, 96)
        costs = [(off[t + 1] - off[t]) ** 2 for t in range(12)]  # cells x steps, steps ~ cells
        mine = decomp.shard_tubes(costs, world)[rank]
        out = {t: oracle.run_1d(oracle.SYS_EULER1D, U[:, off[t]:off[t + 1]], dx[t], t_end=0.02, cfl=0.5,
                                bc=(1, 1))[0] for t in mine}
        parts = [None] * world
        dist.all_gather_object(parts, out)
        if rank == 0:
            got = {k: v for p in parts for k, v in p.items()}
            assert sorted(got) == list(range(12))
            for t in range(12):
                ref = oracle.run_1d(oracle.SYS_EULER1D, U[:, off[t]:off[t + 1]], dx[t], t_end=0.02, cfl=0.5,
                                    bc=(1, 1))[0]
                assert np.array_equal(got[t], ref)
    finally:
        dist.destroy_process_group()


def test_tube_sharding_gathers_every_tube_once():
    """Tubes sharded by cost over 3 gloo ranks, each run where it landed, the
    gather (the only collective) returns every tube once and unchanged."""
    mp.spawn(_worker_tubes, args=(3, _free_port()), nprocs=3, join=True)


def test_shard_tubes_balance():
    rng = np.random.default_rng(5)
    for world in (1, 2, 3, 8):
        costs = rng.integers(256, 8192, 500).astype(float) ** 2
        shards = decomp.shard_tubes(costs, world)
        flat = sorted(t for s in shards for t in s)
        assert flat == list(range(500))
        loads = [costs[s].sum() for s in shards]
        assert max(loads) <= costs.sum() / world + costs.max()
