"""TENO7-ext (the extended seventh-order TENO reconstruction with neighbour-face
shock detection, Sec. 3) for hyperbolic conservation laws on GB300, behind the
C ABI of libteno7 (include/teno7.h).

Modules:
  binding  ctypes marshalling of the C ABI (Context: one grid and precision
           bound to a CUDA stream); no arithmetic happens in Python
  build    compiles libteno7.so for sm_103a in-tree
  adjoint  torch.autograd.Function over checkpointed RK3 steps (the adjoint
           kernels of the library)
  decomp   host logic of slab decomposition and batch sharding across ranks
  adr      approximate dispersion relation of the schemes (Pirozzoli's
           procedure), with the right-hand sides evaluated by t7_euler_rhs
  inputs   seeded initial data of the paper's cases and the synthetic workloads

Example: Shu-Osher on 1600 cells to t = 1.8 in FP32 (device-side CFL steps)::

    import torch
    from paper_1808_00037_gb300 import binding as B, inputs as I

    U, dx = I.shu_osher(1600)                       # [3][1600] (rho, rho u, E)
    ctx = B.Context(B.T7_EULER1D, 1600, dx, prec=B.T7_F32, bc=(1, 1, 0, 0))
    Ug = torch.tensor(U, dtype=torch.float32, device="cuda")
    steps, t = ctx.run(Ug, 0.5, t_end=1.8)          # Ug advanced in place
"""
