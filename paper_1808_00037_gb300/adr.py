"""Approximate dispersion relation (ADR) of the nonlinear schemes, the
analysis of Sec. "Approximate dispersion relation analysis" (Pirozzoli's
procedure for nonlinear schemes, in its short-time form).

For the scalar advection u_t + a u_x = 0 (a = 1) on a periodic grid of N
points, each mode n = 1 .. N/2 with reduced wavenumber phi_n = 2 pi n / N is
sampled as u_j = cos(phi_n j); the right-hand side L(u) of the scheme is
evaluated by the CUDA library (t7_euler_rhs), and its Fourier coefficient at
n defines the modified wavenumber

    Phi(phi_n) = i dx L^_n / (a u^_n),

whose real part is the dispersion and imaginary part the dissipation of the
scheme at that wavenumber (Phi = phi for the exact derivative).  For a linear
scheme with upwind face value f^_{j+1/2} = sum_t c_t u_{j+t+o} this is the
closed form -i (1 - e^{-i phi}) sum_t c_t e^{i phi (t+o)}; for the nonlinear
schemes the stencil selection depends on the wave, which is the point of the
analysis.  The Fourier coefficients are taken with torch.fft on the device.
"""
from __future__ import annotations

import math

import numpy as np

from . import binding as B


def adr(n_points: int = 256, *, scheme: int = B.T7_TENO7EXT, prec: int = B.T7_F64, CT: float = 1e-5,
        eps: float = -1.0):
    """Returns (phi[N/2], Phi[N/2] complex) for modes n = 1 .. N/2 on [0, 1)."""
    import torch
    N = int(n_points)
    if N < 8 or N % 2:
        raise ValueError("n_points must be even and >= 8")
    dx = 1.0 / N
    ctx = B.Context(B.T7_SCALAR_ADVECTION, N, dx, prec=prec, bc=(B.T7_BC_PERIODIC,) * 4, adv_speed=1.0, CT=CT,
                    eps_x=eps, scheme=scheme)
    j = torch.arange(N, dtype=torch.float64, device="cuda")
    modes = torch.arange(1, N // 2 + 1, dtype=torch.float64, device="cuda")
    phi = 2.0 * math.pi * modes / N
    U = torch.cos(phi[:, None] * j[None, :]).to(ctx.dtype).contiguous()  # [N/2, N]
    L = torch.empty_like(U)
    for k in range(N // 2):
        ctx.euler_rhs(U[k:k + 1], out=L[k:k + 1])
    ctx.sync()
    idx = torch.arange(N // 2, device="cuda")
    Lh = torch.fft.fft(L.double(), dim=1)[idx, idx + 1]
    Uh = torch.fft.fft(U.double(), dim=1)[idx, idx + 1]
    Phi = 1j * dx * Lh / Uh
    return phi.cpu().numpy(), Phi.cpu().numpy()


def resolving_wavenumber(phi, Phi, tol: float) -> float:
    """Largest phi_n below which |Phi - phi| stays under tol (the scheme's
    resolving efficiency at that tolerance, as a reduced wavenumber)."""
    bad = np.nonzero(np.abs(Phi - phi) > tol)[0]
    return float(phi[-1] if bad.size == 0 else (phi[bad[0] - 1] if bad[0] > 0 else 0.0))
