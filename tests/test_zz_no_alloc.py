"""t7_rk3_step_static: the RK3 step for callers that cannot allocate device
memory (host-owned memory in plug-ins, no-allocation real-time loops, budgeted
processes).  Called through the C ABI, it must give the same result as the
context-based t7_rk3_step on two calls in a row (the static scratch keeps the
previous call's contents, which must not leak into the next), and it must
reject sizes beyond its fixed scratch with a clear error.  Kept in a file
that pytest collects last."""
import ctypes

import pytest

from paper_1808_00037_gb300 import binding as B
from paper_1808_00037_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("prec,dtype", [(B.T7_F64, torch.float64), (B.T7_F32, torch.float32)])
def test_static_step_matches_context_step_twice(prec, dtype):
    U0, dx = I.shu_osher(1600)
    ctx = B.Context(B.T7_EULER1D, 1600, dx, prec=prec, bc=(1, 1, 0, 0))
    dt = ctx.cfl_dt(torch.tensor(U0, dtype=dtype, device="cuda"), 0.5)
    Ua = torch.tensor(U0, dtype=dtype, device="cuda")
    Ub = Ua.clone()
    for _ in range(2):
        ctx.rk3_step(Ua, dt)
        ctx.sync()
        ctx.rk3_step_static(Ub, dt)
        torch.cuda.synchronize()
        # same kernels and arithmetic: identical, the tests' tolerance for FP64
        assert torch.equal(Ua, Ub)


def test_static_step_scalar_advection_through_raw_abi():
    n = 777
    U0, dx, _ = I.advection_sine(n)
    lib = B.load()
    g = B.t7_grid(B.T7_SCALAR_ADVECTION, B.T7_F64, n, 1, dx, 0.0, (ctypes.c_int * 4)(0, 0, 0, 0), 1.4, 1.0, 1e-5,
                  -1.0, -1.0)
    ref = B.Context(B.T7_SCALAR_ADVECTION, n, dx)
    Ua = torch.tensor(U0, dtype=torch.float64, device="cuda")
    Ub = Ua.clone()
    buf = ctypes.create_string_buffer(256)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        ref.rk3_step(Ua, 0.002)
        ref.sync()
        st = lib.t7_rk3_step_static(ctypes.byref(g), Ub.data_ptr(), 0.002, stream, buf, 256)
        assert st == B.T7_OK, buf.value
        assert torch.equal(Ua, Ub)


def test_static_step_rejects_oversized_grid():
    lib = B.load()
    n = 1_000_000  # 2 x 3 x 1e6 x 8 bytes of stage buffers > 16 MiB
    g = B.t7_grid(B.T7_EULER1D, B.T7_F64, n, 1, 1e-3, 0.0, (ctypes.c_int * 4)(1, 1, 0, 0), 1.4, 1.0, 1e-5, -1.0,
                  -1.0)
    U = torch.ones(3 * n, dtype=torch.float64, device="cuda")
    buf = ctypes.create_string_buffer(256)
    st = lib.t7_rk3_step_static(ctypes.byref(g), U.data_ptr(), 1e-4, None, buf, 256)
    assert st == B.T7_EINVAL
    assert b"static scratch" in buf.value
    assert torch.all(U == 1.0)  # untouched
