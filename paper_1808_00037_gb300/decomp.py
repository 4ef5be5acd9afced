"""Slab decompositions of the 1D and 2D schemes over ranks (torch.distributed),
tube sharding for ragged batches, and FP64 domain sums.

Rank r owns the contiguous cells [lo_r, hi_r) of a 1D domain.  Every RHS
evaluation needs, per side, a halo of HALO = 4 cells and the global
Lax-Friedrichs alpha: the RHS at cell i reads faces i-1/2 and i+1/2, whose
polynomials reach cells i-4 .. i+4 and whose neighbour-face cutoff bits are
computed from windows inside the same range.  So one SSP-RK3 stage is

    exchange 4-cell halos  ->  all-reduce(max) of the local alphas
    ->  RHS of the padded slab (inner cells only)  ->  RK combination,

and each step starts with an all-reduce(max) for the CFL step.  The domain's
own boundaries (periodic or zero-gradient) become halos from the periodic
neighbour or copies of the edge cell.  These are the only exchanges: the path
has no other collective.

The per-rank RHS is a callable ``rhs(U_padded, alpha) -> L(U) on the padded
slab`` so the same exchange logic drives any implementation; the CPU tests
run it with the oracle on gloo ranks and require bit-identical results to
the unsplit run.
"""
from __future__ import annotations

import numpy as np

HALO = 4


def partition(n: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous cell range [lo, hi) of `rank` (sizes differ by at most one)."""
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def exchange_halos(U, periodic: bool):
    """U: [m, n_local] numpy (1D), or [4, ny_local, nx] (2D, split along y).
    Returns the array padded by HALO cells (rows) on each side of axis 1, the
    halos coming from the neighbouring ranks (or from the domain boundary
    condition at the ends: periodic wrap, or copies of the edge cell/row)."""
    import torch
    import torch.distributed as dist

    world, rank = dist.get_world_size(), dist.get_rank()
    n = U.shape[1]
    if n < HALO:
        raise ValueError("each rank needs at least 4 cells (rows)")
    left_n = (rank - 1) % world if (periodic or rank > 0) else None
    right_n = (rank + 1) % world if (periodic or rank < world - 1) else None
    send_l = torch.from_numpy(np.ascontiguousarray(U[:, :HALO]))
    send_r = torch.from_numpy(np.ascontiguousarray(U[:, -HALO:]))
    recv_l = torch.empty(send_l.shape, dtype=torch.float64)
    recv_r = torch.empty(send_r.shape, dtype=torch.float64)
    reqs = []
    if world > 1:
        # tags by direction: with two ranks (periodic) both neighbours are the
        # same rank, and the two messages must not be confused
        LEFTWARD, RIGHTWARD = 1, 2
        if left_n is not None:
            reqs.append(dist.isend(send_l, left_n, tag=LEFTWARD))
            reqs.append(dist.irecv(recv_l, left_n, tag=RIGHTWARD))
        if right_n is not None:
            reqs.append(dist.isend(send_r, right_n, tag=RIGHTWARD))
            reqs.append(dist.irecv(recv_r, right_n, tag=LEFTWARD))
        for r in reqs:
            r.wait()
    else:
        if periodic:
            recv_l, recv_r = send_r.clone(), send_l.clone()
    shape = list(U.shape)
    shape[1] = n + 2 * HALO
    P = np.empty(shape)
    P[:, HALO:HALO + n] = U
    P[:, :HALO] = recv_l.numpy() if left_n is not None else U[:, :1]
    P[:, HALO + n:] = recv_r.numpy() if right_n is not None else U[:, -1:]
    return P


def allreduce_max(x):
    """Max over ranks of a float, or element-wise of a tuple of floats."""
    import torch
    import torch.distributed as dist

    t = torch.tensor(np.atleast_1d(np.asarray(x, np.float64)))
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0]) if np.ndim(x) == 0 else tuple(float(v) for v in t)


def global_sums(U_local):
    """Domain sums of each conserved variable over all ranks, in FP64 (the
    conservation check of a decomposed run): sum over the rank's cells, then
    an all-reduce(sum)."""
    import torch
    import torch.distributed as dist

    U = np.asarray(U_local, np.float64)
    t = torch.from_numpy(U.reshape(U.shape[0], -1).sum(axis=1).copy())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.numpy()


def shard_tubes(costs, world: int):
    """Independent tubes to ranks by cost (e.g. cells x steps): longest
    processing time first, each tube to the currently least-loaded rank.
    Returns one list of tube indices per rank; the largest load is at most
    (4/3 - 1/(3 world)) times the optimum and below mean + max cost."""
    order = np.argsort(-np.asarray(costs, np.float64), kind="stable")
    loads = np.zeros(world)
    out = [[] for _ in range(world)]
    for t in order:
        r = int(np.argmin(loads))
        out[r].append(int(t))
        loads[r] += costs[t]
    return out


def rk3_run(U_local, rhs, alpha_local, *, dx: float, cfl: float, t_end: float, max_steps: int, periodic: bool):
    """March the local slab with the SSP-RK3 scheme, exchanging halos and the
    global alpha at every stage.  rhs(P, alpha) -> L on the padded slab P;
    alpha_local(U) -> max characteristic speed of the rank's cells.  Returns
    (U_local, steps, t); every rank takes the same steps and dt."""
    def L(U, alpha):
        return rhs(exchange_halos(U, periodic), alpha)[:, HALO:-HALO]

    U = np.array(U_local, dtype=np.float64)
    t, steps = 0.0, 0
    while steps < max_steps and t < t_end:
        a0 = allreduce_max(alpha_local(U))
        dt = (cfl * dx) / a0
        if t + dt > t_end:
            dt = t_end - t
        U0 = U.copy()
        U1 = U0 + dt * L(U0, a0)
        a1 = allreduce_max(alpha_local(U1))
        U2 = 0.75 * U0 + 0.25 * (U1 + dt * L(U1, a1))
        a2 = allreduce_max(alpha_local(U2))
        U = (1.0 / 3.0) * U0 + (2.0 / 3.0) * (U2 + dt * L(U2, a2))
        t = t + dt
        steps += 1
    return U, steps, t


def rk3_run_2d(U_local, rhs, alpha_local, *, dx: float, dy: float, cfl: float, t_end: float, max_steps: int,
               periodic_y: bool):
    """2D slab decomposition along y (rows stay contiguous): U_local
    [4, ny_local, nx].  rhs(P, (ax, ay)) -> L on the padded slab P (4 halo rows
    per side; x boundaries inside the rank); alpha_local(U) -> (ax, ay) of the
    rank's cells.  Per stage: halo-row exchange and all-reduce(max) of both
    alphas; per step the CFL step cfl / (ax/dx + ay/dy).  Returns
    (U_local, steps, t)."""
    def L(U, a):
        return rhs(exchange_halos(U, periodic_y), a)[:, HALO:-HALO]

    U = np.array(U_local, dtype=np.float64)
    t, steps = 0.0, 0
    while steps < max_steps and t < t_end:
        a0 = allreduce_max(alpha_local(U))
        dt = cfl / (a0[0] / dx + a0[1] / dy)
        if t + dt > t_end:
            dt = t_end - t
        U0 = U.copy()
        U1 = U0 + dt * L(U0, a0)
        a1 = allreduce_max(alpha_local(U1))
        U2 = 0.75 * U0 + 0.25 * (U1 + dt * L(U1, a1))
        a2 = allreduce_max(alpha_local(U2))
        U = (1.0 / 3.0) * U0 + (2.0 / 3.0) * (U2 + dt * L(U2, a2))
        t = t + dt
        steps += 1
    return U, steps, t
