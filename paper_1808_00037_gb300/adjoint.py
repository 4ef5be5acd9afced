"""Gradients through SSP-RK3 runs of the 1D Euler TENO7-ext scheme.

``CheckpointedRK3`` is a ``torch.autograd.Function``: its forward advances a
state by ``nsteps`` SSP-RK3 steps of fixed size dt with the CUDA stage kernels
(``t7_rk3_step``), keeping the state every ``every`` steps; its backward
replays each segment from its checkpoint with recorded steps
(``t7_rk3_step_record``: stage states, forward stencil codes and alphas go to
a tape) and maps the incoming gradient back step by step with the
hand-written discrete adjoint of each recorded step
(``t7_rk3_step_adjoint_recorded``: ``(dL/dU)^T`` applied by the adjoint kernel
with the recorded selection and alpha frozen, accumulated straight into the
RK3 adjoint buffers).  Memory: the checkpoints plus one segment of states and
tape entries.

``sine_modes_gradient`` sets up the adjoint benchmark problem -- periodic [0,1),
rho0 = 1 + sum_k a_k sin(2 pi k x), u0 = p0 = 1, J = sum_i rho_i^2 dx at the
final time -- and returns J and dJ/da through the Function above.  The initial
condition, J and their derivatives are the problem's set-up (PyTorch tensor
arithmetic); every step of the scheme and of its adjoint runs in the CUDA
library.
"""
from __future__ import annotations

import math

import numpy as np

from . import binding as B


def _torch():
    import torch
    return torch


class CheckpointedRK3:
    """Namespace holding the autograd Function (created lazily with torch)."""

    _fn = None

    @classmethod
    def apply(cls, U0, context: "B.Context", dt: float, nsteps: int, every: int = 100):
        if cls._fn is None:
            cls._fn = _make_function()
        return cls._fn.apply(U0, context, dt, nsteps, every)


def _make_function():
    torch = _torch()

    class _RK3(torch.autograd.Function):
        @staticmethod
        def forward(fctx, U0, context, dt, nsteps, every):
            U = U0.detach().contiguous().clone()
            cps = [U.clone()]
            for s in range(nsteps):
                context.rk3_step(U, dt)
                if (s + 1) % every == 0 and s + 1 < nsteps:
                    cps.append(U.clone())
            context.sync()
            fctx.context, fctx.dt, fctx.nsteps, fctx.every = context, dt, nsteps, every
            fctx.cps = cps
            return U

        @staticmethod
        def backward(fctx, grad_out):
            context, dt, nsteps, every = fctx.context, fctx.dt, fctx.nsteps, fctx.every
            lam = grad_out.detach().contiguous().clone()
            # one segment's states and tape entries, reused for every segment
            states = [torch.empty_like(fctx.cps[0]) for _ in range(every + 1)]
            tapes = torch.empty((every, context.tape_bytes()), dtype=torch.uint8, device=lam.device)
            for seg in reversed(range(len(fctx.cps))):
                start = seg * every
                count = min(start + every, nsteps) - start
                states[0].copy_(fctx.cps[seg])
                for s in range(count):
                    context.rk3_step_record(states[s], states[s + 1], dt, tapes[s])
                for s in reversed(range(count)):
                    context.rk3_step_adjoint_recorded(states[s], tapes[s], dt, lam)
            context.sync()
            return lam, None, None, None, None

    return _RK3


def sine_modes_state(a, n: int, gamma: float = 1.4):
    """U0[3, n] (torch, differentiable in a) of rho0 = 1 + sum a_k sin(2 pi k x),
    u0 = 1, p0 = 1 on periodic [0, 1)."""
    torch = _torch()
    x = (torch.arange(n, dtype=torch.float64, device=a.device) + 0.5) / n
    k = torch.arange(1, a.numel() + 1, dtype=torch.float64, device=a.device)
    S = torch.sin(2 * math.pi * torch.outer(x, k))
    rho = 1.0 + S @ a
    return torch.stack([rho, rho * 1.0, torch.full_like(rho, 1.0 / (gamma - 1.0)) + 0.5 * rho])


def sine_modes_gradient(a_k, n: int = 4096, nsteps: int = 2000, every: int = 100, prec: int = B.T7_F64,
                        cfl: float = 0.5, dt: float | None = None, a_ref=None):
    """J(a) and dJ/da for the sine-mode problem.  dt is held fixed for all a
    (computed once with CFL `cfl` from the state at a_ref, default a) so that
    finite differences and the adjoint differentiate the same discrete map."""
    torch = _torch()
    dtype = torch.float64 if prec == B.T7_F64 else torch.float32
    a = torch.tensor(np.asarray(a_k, np.float64), device="cuda", requires_grad=True)
    ctx = B.Context(B.T7_EULER1D, n, 1.0 / n, prec=prec, bc=(0, 0, 0, 0))
    if dt is None:
        ref = torch.tensor(np.asarray(a_k if a_ref is None else a_ref, np.float64), device="cuda")
        dt = ctx.cfl_dt(sine_modes_state(ref, n).to(dtype).contiguous(), cfl)
    U0 = sine_modes_state(a, n).to(dtype)
    U = CheckpointedRK3.apply(U0, ctx, dt, nsteps, every)
    J = (U[0].double() ** 2).sum() / n
    J.backward()
    return float(J.item()), a.grad.detach().cpu().numpy(), dt


def sine_modes_objective(a_k, n: int, nsteps: int, dt: float, prec: int = B.T7_F64) -> float:
    """J(a) by a plain forward run (for finite differences)."""
    torch = _torch()
    dtype = torch.float64 if prec == B.T7_F64 else torch.float32
    ctx = B.Context(B.T7_EULER1D, n, 1.0 / n, prec=prec, bc=(0, 0, 0, 0))
    a = torch.tensor(np.asarray(a_k, np.float64), device="cuda")
    U = sine_modes_state(a, n).to(dtype).contiguous()
    for _ in range(nsteps):
        ctx.rk3_step(U, dt)
    ctx.sync()
    return float((U[0].double() ** 2).sum().item() / n)
