"""Oracle backends of the slab decomposition (test infrastructure): the same
stage interface as decomp.CudaSlab, computed by the CPU oracle on CPU
tensors, so the multi-rank orchestration can be checked on gloo ranks."""
import numpy as np
import torch

import oracle
from paper_1808_00037_gb300 import decomp


def _np(t):
    return t.detach().cpu().numpy()


def _rk(k, u, u0, dt, L):
    """The Shu-Osher stages in the oracle's expression order."""
    if k == 0:
        return u + dt * L
    if k == 1:
        return 0.75 * u0 + 0.25 * (u + dt * L)
    return (1.0 / 3.0) * u0 + (2.0 / 3.0) * (u + dt * L)


class OracleSlab1D:
    stream = None

    def __init__(self, sys_, dx):
        self.sys, self.dx = sys_, dx

    def alpha(self, P, out):
        out[0] = oracle.alpha_1d(self.sys, _np(decomp.interior(P)))

    def stage(self, k, Us, U0, out, alpha, dt, alpha_out):
        # the oracle's RHS of the padded slab (its own boundary treatment only
        # touches cells outside the interior, whose values are not used)
        L = oracle.rhs_1d(self.sys, _np(Us), self.dx, bc=(1, 1), alpha=float(alpha[0]))[0][:, decomp.HALO:-decomp.HALO]
        u0 = None if U0 is None else _np(decomp.interior(U0))
        decomp.interior(out).copy_(torch.from_numpy(_rk(k, _np(decomp.interior(Us)), u0, dt, L)))
        if alpha_out is not None:
            self.alpha(out, alpha_out)


class OracleSlab2D:
    """2D slab split along y ([4, ny + 8, nx] padded arrays); x boundaries
    inside the slab with codes bcx."""
    stream = None

    def __init__(self, dx, dy, bcx):
        self.dx, self.dy, self.bcx = dx, dy, bcx

    def alpha(self, P, out):
        ax, ay = oracle.alpha_2d(_np(decomp.interior(P)))
        out[0], out[1] = ax, ay

    def stage(self, k, Us, U0, out, alpha, dt, alpha_out):
        a = (float(alpha[0]), float(alpha[1]))
        L = oracle.rhs_2d(_np(Us), self.dx, self.dy, bc=(self.bcx[0], self.bcx[1], 1, 1), alpha=a)[0]
        L = L[:, decomp.HALO:-decomp.HALO]
        u0 = None if U0 is None else _np(decomp.interior(U0))
        decomp.interior(out).copy_(torch.from_numpy(_rk(k, _np(decomp.interior(Us)), u0, dt, L)))
        if alpha_out is not None:
            self.alpha(out, alpha_out)

