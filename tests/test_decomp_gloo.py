"""Multi-rank path on CPU: the slab decomposition of paper_1808_00037_gb300.decomp
(4-cell halo exchange and all-reduce(max) of alpha per RK stage, the CFL step
from the all-reduced alpha) on gloo ranks -- and, in one process, over
several slabs -- each slab's stages computed by the oracle backend of
tests/slab_backends.py.  The gathered result must be bit-identical to the
unsplit oracle run, which pins the halo width, the boundary handling at the
domain ends and the synchronisation of alpha and dt.  The GPU counterpart
(the CUDA slab stages) is tests/test_gpu_slabs.py."""
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_1808_00037_gb300 import decomp
from paper_1808_00037_gb300 import inputs as I
from slab_backends import OracleSlab1D, OracleSlab2D


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
        slab = decomp.Slab(OracleSlab1D(oracle.SYS_EULER1D, dx), U[:, lo:hi])
        steps, t = decomp.rk3_run_slabs(decomp.RankSlabs(slab, periodic), decomp.cfl_dt_1d(dx, 0.5),
                                        t_end=t_end, max_steps=max_steps)
        parts = [None] * world
        dist.all_gather_object(parts, (lo, hi, slab.state().numpy().copy(), steps, t))
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


@pytest.mark.parametrize("nslabs", [1, 2, 3])
@pytest.mark.parametrize("name", ["sod", "smooth-periodic"])
def test_local_slabs_bit_identical(nslabs, name):
    """All slabs in one process (the one-GPU layout, here on CPU tensors): the
    same orchestration with device-local halo copies and a max over the slabs
    as the all-reduce; bit-identical to the unsplit oracle run."""
    U, dx, periodic, t_end, max_steps = _case(name)
    bc = (0, 0) if periodic else (1, 1)
    slabs = [decomp.Slab(OracleSlab1D(oracle.SYS_EULER1D, dx), U[:, lo:hi])
             for lo, hi in (decomp.partition(U.shape[1], nslabs, r) for r in range(nslabs))]
    steps, t = decomp.rk3_run_slabs(decomp.LocalSlabs(slabs, periodic), decomp.cfl_dt_1d(dx, 0.5),
                                    t_end=min(t_end, 0.02), max_steps=min(max_steps, 12))
    Uo, so, to, _ = oracle.run_1d(oracle.SYS_EULER1D, U, dx, t_end=min(t_end, 0.02), cfl=0.5, bc=bc,
                                  max_steps=min(max_steps, 12))
    assert (steps, t) == (so, to)
    assert np.array_equal(np.concatenate([s.state().numpy() for s in slabs], axis=1), Uo)


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
        slab = decomp.Slab(OracleSlab2D(dx, dy, bcx), U[:, lo:hi], nalpha=2)
        steps, t = decomp.rk3_run_slabs(decomp.RankSlabs(slab, periodic), decomp.cfl_dt_2d(dx, dy, 0.4),
                                        t_end=np.inf, max_steps=nsteps)
        Ul = slab.state().numpy().copy()
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
