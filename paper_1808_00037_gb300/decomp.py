"""Slab decompositions of the 1D and 2D schemes, tube sharding for ragged
batches, and FP64 domain sums.

A domain of N cells (2D: N rows, split along y so rows stay contiguous) is cut
into contiguous slabs, one per rank -- or, on one GPU, one per CUDA stream.
Every RHS evaluation of a slab needs, per side, a halo of HALO = 4 cells
(rows) and the global Lax-Friedrichs alpha: the RHS at cell i reads faces
i-1/2 and i+1/2, whose polynomials reach cells i-4 .. i+4 and whose
neighbour-face cutoff bits are computed from windows inside the same range
(Eq. app, Eq. vec).  So one SSP-RK3 stage is

    fill the 4-cell halos  ->  stage kernel on the padded slab
    ->  all-reduce(max) of the slabs' alphas of the stage output,

and the step's CFL step comes from the all-reduced alpha of U^n.  The
domain's own boundaries (periodic or zero-gradient) become halos from the
periodic neighbour or copies of the edge cell.  These are the only
exchanges: the path has no other collective.

Each slab keeps its three RK states (U^n and the two stage states) as arrays
padded by HALO cells (rows) on each side of axis 1, so the stage kernel reads
its halos in place.  A slab's ``backend`` does the arithmetic:
``alpha(P, out)`` (local max wave speed into a one-element float64 tensor)
and ``stage(k, Us, U0, out, alpha, dt, alpha_out)`` (one Shu-Osher stage).
``CudaSlab`` wraps the library's t7_slab_* entry points, so the RK stages,
the wave-speed reductions and the alpha values never leave the GPU; only dt
(one double per step) is read on the host.
"""
from __future__ import annotations

import numpy as np

HALO = 4


def partition(n: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous cell range [lo, hi) of `rank` (sizes differ by at most one)."""
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def padded(U_local):
    """U_local [m, n] (or [4, ny, nx]) as a tensor padded by HALO cells (rows)
    on each side of axis 1, halos zero."""
    import torch

    t = U_local if isinstance(U_local, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(U_local))
    shape = list(t.shape)
    shape[1] += 2 * HALO
    P = torch.zeros(shape, dtype=t.dtype, device=t.device)
    P[:, HALO:-HALO] = t
    return P


def interior(P):
    return P[:, HALO:-HALO]


class CudaSlab:
    """A slab backend on the CUDA library: one context per slab (1D: nx = the
    slab's cells; 2D: nx columns, ny = the slab's rows), t7_slab_alpha /
    t7_slab_stage on padded tensors (2D: alpha_x and alpha_y, two doubles)."""

    def __init__(self, ctx):
        self.ctx = ctx
        self.stream = ctx.stream

    def alpha(self, P, out):
        self.ctx.slab_alpha(P, out)

    def stage(self, k, Us, U0, out, alpha, dt, alpha_out):
        self.ctx.slab_stage(k, Us, U0, out, alpha, dt, alpha_out)


class Slab:
    """One slab: its backend, its three padded RK states and its local alphas."""

    def __init__(self, backend, U_local, nalpha: int = 1):
        import torch

        self.backend = backend
        self.stream = getattr(backend, "stream", None)
        self.P = [padded(U_local)]
        self.P += [torch.zeros_like(self.P[0]) for _ in range(2)]
        self.a = [torch.zeros(nalpha, dtype=torch.float64, device=self.P[0].device) for _ in range(3)]

    def state(self):
        return interior(self.P[0])


class LocalSlabs:
    """Every slab of the domain in this process, in domain order (one GPU,
    one CUDA stream per slab, or CPU tensors): halos are device-local copies
    and the all-reduce is a max over the slabs' values.  Work on the slabs'
    streams is ordered through the current stream at each all-reduce."""

    def __init__(self, slabs, periodic: bool):
        self.slabs = slabs
        self.periodic = periodic

    def _streams(self):
        return [s.stream for s in self.slabs if s.stream is not None]

    def fill_halos(self, k: int):
        import torch

        n = len(self.slabs)
        for i, s in enumerate(self.slabs):
            P = s.P[k]
            left = self.slabs[i - 1].P[k] if (i > 0 or self.periodic) else None
            right = self.slabs[(i + 1) % n].P[k] if (i < n - 1 or self.periodic) else None
            ctx = torch.cuda.stream(s.stream) if s.stream is not None else _null()
            with ctx:
                if s.stream is not None:
                    for j in (i - 1, (i + 1) % n):
                        if self.slabs[j].stream is not None and j != i:
                            s.stream.wait_stream(self.slabs[j].stream)
                P[:, :HALO].copy_(left[:, -2 * HALO:-HALO] if left is not None else
                                  P[:, HALO:HALO + 1].expand_as(P[:, :HALO]))
                P[:, -HALO:].copy_(right[:, HALO:2 * HALO] if right is not None else
                                   P[:, -HALO - 1:-HALO].expand_as(P[:, -HALO:]))

    def allreduce_max(self, k: int, out):
        """out <- max over the slabs of their alpha slot k; every slab's stream
        then waits for it."""
        import torch

        streams = self._streams()
        cur = torch.cuda.current_stream() if streams else None
        for st in streams:
            cur.wait_stream(st)
        torch.amax(torch.stack([s.a[k] for s in self.slabs]), dim=0, out=out)
        for st in streams:
            st.wait_stream(cur)
        return out


class RankSlabs:
    """One slab per rank over torch.distributed (NCCL for CUDA tensors, gloo
    for CPU ones): halos travel by point-to-point messages in two phases
    (rightward, then leftward, so that with two periodic ranks the two
    messages between the same pair never cross), the alphas by all-reduce(max)."""

    def __init__(self, slab, periodic: bool):
        import torch.distributed as dist

        self.slabs = [slab]
        self.periodic = periodic
        self.world, self.rank = dist.get_world_size(), dist.get_rank()

    def fill_halos(self, k: int):
        import torch
        import torch.distributed as dist

        P = self.slabs[0].P[k]
        world, rank = self.world, self.rank
        if P.shape[1] < 3 * HALO:
            raise ValueError("each rank needs at least 4 cells (rows)")
        left = (rank - 1) % world if (self.periodic or rank > 0) else None
        right = (rank + 1) % world if (self.periodic or rank < world - 1) else None
        if world == 1:
            if self.periodic:
                P[:, :HALO].copy_(P[:, -2 * HALO:-HALO])
                P[:, -HALO:].copy_(P[:, HALO:2 * HALO])
        else:
            RIGHTWARD, LEFTWARD = 1, 2
            for direction in (RIGHTWARD, LEFTWARD):
                src = right if direction == LEFTWARD else left    # who sends to me in this phase
                dst = right if direction == RIGHTWARD else left   # whom I send to
                ops = []
                if dst is not None:
                    edge = P[:, -2 * HALO:-HALO] if direction == RIGHTWARD else P[:, HALO:2 * HALO]
                    ops.append(dist.P2POp(dist.isend, edge.contiguous(), dst, tag=direction))
                recv = None
                if src is not None:
                    recv = torch.empty_like(P[:, :HALO]).contiguous()
                    ops.append(dist.P2POp(dist.irecv, recv, src, tag=direction))
                if ops:
                    for r in dist.batch_isend_irecv(ops):
                        r.wait()
                if recv is not None:
                    (P[:, :HALO] if direction == RIGHTWARD else P[:, -HALO:]).copy_(recv)
        if left is None:
            P[:, :HALO].copy_(P[:, HALO:HALO + 1].expand_as(P[:, :HALO]))
        if right is None:
            P[:, -HALO:].copy_(P[:, -HALO - 1:-HALO].expand_as(P[:, -HALO:]))

    def allreduce_max(self, k: int, out):
        import torch.distributed as dist

        out.copy_(self.slabs[0].a[k])
        dist.all_reduce(out, op=dist.ReduceOp.MAX)
        return out


class _null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


def cfl_dt_1d(dx: float, cfl: float):
    """dt of the 1D CFL condition, in the expression order of the unsplit run."""
    return lambda a: (cfl * dx) / float(a[0])


def cfl_dt_2d(dx: float, dy: float, cfl: float):
    """dt of the 2D CFL condition cfl / (ax/dx + ay/dy)."""
    return lambda a: cfl / (float(a[0]) / dx + float(a[1]) / dy)


def rk3_run_slabs(comm, dt_of_alpha, *, t_end: float, max_steps: int):
    """March every slab of `comm` with the SSP-RK3 scheme (Shu-Osher form):

        U1 = U + dt L(U);  U2 = 3/4 U + 1/4 (U1 + dt L(U1));  U = 1/3 U + 2/3 (U2 + dt L(U2)),

    each stage one backend call per slab after its halos are filled, each L
    with the all-reduced alpha of its input.  dt = dt_of_alpha(alpha(U^n)),
    the last step clipped to land on t_end.  Returns (steps, t); every slab
    takes the same steps and dt."""
    import torch

    slabs = comm.slabs
    dev = slabs[0].P[0].device
    g = [torch.zeros_like(slabs[0].a[0]) for _ in range(3)]  # all-reduced alphas
    cuda = dev.type == "cuda"
    if cuda:
        # the all-reduced alpha of U^n reaches the host through a pinned buffer
        # and an event, so that only the host waits for it
        a_host = torch.empty(g[0].shape, dtype=g[0].dtype, pin_memory=True)
        a_ready = torch.cuda.Event()
    for s in slabs:
        with (torch.cuda.stream(s.stream) if s.stream is not None else _null()):
            s.backend.alpha(s.P[0], s.a[0])
    t, steps = 0.0, 0
    if steps < max_steps and t < t_end:
        comm.allreduce_max(0, g[0])
    while steps < max_steps and t < t_end:
        if cuda:
            a_host.copy_(g[0], non_blocking=True)
            a_ready.record()
        # the halos of U^n do not depend on dt: they are queued before the
        # host waits for it, so the device has them to do meanwhile
        comm.fill_halos(0)
        if cuda:
            a_ready.synchronize()
        dt = dt_of_alpha(a_host if cuda else g[0])
        if t + dt > t_end:
            dt = t_end - t
        for k in range(3):
            if k > 0:
                comm.fill_halos(k)
            for s in slabs:
                Us, U0 = s.P[k], s.P[0]
                out = s.P[k + 1] if k < 2 else s.P[0]
                with (torch.cuda.stream(s.stream) if s.stream is not None else _null()):
                    s.backend.stage(k, Us, None if k == 0 else U0, out, g[k], dt, s.a[(k + 1) % 3])
            if k < 2:
                comm.allreduce_max(k + 1, g[k + 1])
        t = t + dt
        steps += 1
        if steps < max_steps and t < t_end:
            # alpha of U^{n+1}: every slab's stage 2 wrote its part into a[0]
            comm.allreduce_max(0, g[0])
    if any(s.stream is not None for s in slabs):
        cur = torch.cuda.current_stream()
        for s in slabs:
            if s.stream is not None:
                cur.wait_stream(s.stream)
    return steps, t


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

