"""Runs every form of the forward path, the discrete adjoint and the
no-allocation step through the C ABI at ragged and tiny sizes and saves the
results: python tests/checked_driver.py <out.npz>.
The library is the one binding.LIB_PATH names (T7_LIBRARY: the index-checked
build).  Any error status -- a failed index check (T7_EINDEX) above all --
raises.  Used by test_gpu_checked.py, which runs it once with each build."""
import math
import sys
from pathlib import Path

import numpy as np
import torch

sys.path.insert(0, str(Path(__file__).resolve().parents[1]))

from paper_1808_00037_gb300 import binding as B  # noqa: E402
from paper_1808_00037_gb300 import decomp  # noqa: E402
from paper_1808_00037_gb300 import inputs as I  # noqa: E402

DT = {B.T7_F64: torch.float64, B.T7_F32: torch.float32, B.T7_MIXED: torch.float64}
PNAME = {B.T7_F64: "f64", B.T7_F32: "f32", B.T7_MIXED: "mixed"}


def host(t):
    return t.double().cpu().numpy()


def forms_1d(res):
    cases = {
        "euler-shu-osher-759": (B.T7_EULER1D, *I.shu_osher(1600)[:2], (1, 1)),
        "euler-smooth-3": (B.T7_EULER1D, *I.random_euler_smooth(9, 3)[:2], (0, 0)),
        "euler-smooth-61": (B.T7_EULER1D, *I.random_euler_smooth(10, 61)[:2], (0, 0)),
        "euler-sod-122": (B.T7_EULER1D, *I.riemann_tube(122, *I.SOD)[:2], (1, 1)),
        "advection-200": (B.T7_SCALAR_ADVECTION, *I.advection_sine(200)[:2], (0, 0)),
        "burgers-97": (B.T7_BURGERS, *I.burgers_sine(97)[:2], (0, 0)),
    }
    for name, (sysid, U, dx, bc) in cases.items():
        if name == "euler-shu-osher-759":
            U = np.ascontiguousarray(U[:, :759])
        for prec in (B.T7_F64, B.T7_F32, B.T7_MIXED):
            for scheme in (B.T7_TENO7EXT, B.T7_TENO5):
                if scheme == B.T7_TENO5 and prec == B.T7_MIXED:
                    continue
                tag = f"1d-{name}-{PNAME[prec]}-s{scheme}"
                c = B.Context(sysid, U.shape[1], dx, prec=prec, bc=bc + (0, 0), gamma=1.4, scheme=scheme)
                Ug = torch.tensor(U, dtype=DT[prec], device="cuda")
                L, m = c.euler_rhs(Ug, want_masks=True)
                res[tag + "-rhs"], res[tag + "-masks"] = host(L), m.cpu().numpy()
                steps, t = c.run(Ug, 0.5, max_steps=6)
                res[tag + "-run"] = host(Ug)
                c.close()
    # host-array runs: the parted last stage (FP32, FP64)
    U, dx = I.shu_osher(1600)
    for prec in (B.T7_F64, B.T7_F32):
        c = B.Context(B.T7_EULER1D, 1600, dx, prec=prec, bc=(1, 1, 0, 0), gamma=1.4)
        Uh = torch.tensor(U, dtype=DT[prec]).pin_memory()
        c.run_host(Uh, 0.5, max_steps=3)
        res[f"1d-run-host-{PNAME[prec]}"] = Uh.double().numpy()
        c.close()
    # per-field alphas
    U, dx, _ = I.random_euler_smooth(11, 301)
    for prec in (B.T7_F64, B.T7_F32):
        c = B.Context(B.T7_EULER1D, 301, dx, prec=prec, bc=(0, 0, 0, 0), gamma=1.4,
                      alpha_mode=B.T7_ALPHA_PER_FIELD)
        Ug = torch.tensor(U, dtype=DT[prec], device="cuda")
        c.run(Ug, 0.5, max_steps=5)
        res[f"1d-per-field-{PNAME[prec]}"] = host(Ug)
        c.close()


def adjoint_and_static(res):
    """The discrete adjoint (RHS, RK3 step, recorded step) and the
    no-allocation step, periodic and zero-gradient."""
    for name, (U, dx), bc in (("smooth-301", I.random_euler_smooth(9, 301)[:2], (0, 0)),
                              ("sod-122", I.riemann_tube(122, *I.SOD)[:2], (1, 1))):
        v = np.random.default_rng(1).standard_normal(U.shape)
        for prec in (B.T7_F64, B.T7_F32):
            tag = f"adj-{name}-{PNAME[prec]}"
            c = B.Context(B.T7_EULER1D, U.shape[1], dx, prec=prec, bc=bc + (0, 0), gamma=1.4)
            Ug = torch.tensor(U, dtype=DT[prec], device="cuda")
            vg = torch.tensor(v, dtype=DT[prec], device="cuda")
            dt = 0.2 * dx
            res[tag + "-rhs"] = host(c.euler_rhs_adjoint(Ug, vg))
            lam = vg.clone()
            res[tag + "-step"] = host(c.rk3_step_adjoint(Ug, dt, lam))
            tape = torch.empty(c.tape_bytes(), dtype=torch.uint8, device="cuda")
            U1 = torch.empty_like(Ug)
            res[tag + "-recorded-U"] = host(c.rk3_step_record(Ug, U1, dt, tape))
            lam = vg.clone()
            res[tag + "-recorded"] = host(c.rk3_step_adjoint_recorded(Ug, tape, dt, lam))
            c.sync()
            Us = Ug.clone()
            res[tag + "-static"] = host(c.rk3_step_static(Us, dt))
            c.close()


def slabs_1d(res):
    U, dx = I.shu_osher(1600)
    U = np.ascontiguousarray(U[:, :797])
    for prec in (B.T7_F64, B.T7_F32, B.T7_MIXED):
        slabs = []
        for r in range(3):
            lo, hi = decomp.partition(U.shape[1], 3, r)
            ctx = B.Context(B.T7_EULER1D, hi - lo, dx, prec=prec, gamma=1.4, stream=torch.cuda.Stream())
            slabs.append(decomp.Slab(decomp.CudaSlab(ctx), torch.tensor(U[:, lo:hi], dtype=DT[prec], device="cuda")))
        torch.cuda.synchronize()
        comm = decomp.LocalSlabs(slabs, False)
        decomp.rk3_run_slabs(comm, decomp.cfl_dt_1d(dx, 0.5), t_end=math.inf, max_steps=4)
        torch.cuda.synchronize()
        res[f"1d-slabs-{PNAME[prec]}"] = np.concatenate([host(s.state()) for s in slabs], axis=1)


def batch(res):
    sizes = [3, 40, 300, 777, 1000]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    parts, dx = [], []
    for n in sizes:
        Ut, dxt = I.riemann_tube(n, *I.SOD)[:2]
        parts.append(Ut)
        dx.append(dxt)
    U = np.ascontiguousarray(np.concatenate(parts, axis=1))
    for prec in (B.T7_F64, B.T7_F32):
        for g in (1, 8):
            c = B.Context(B.T7_EULER1D, int(off[-1]), 1.0, prec=prec, gamma=1.4)
            Ug = torch.tensor(U, dtype=DT[prec], device="cuda")
            steps, t = c.batch_run(Ug, off, np.array(dx), 0.05, 0.5, group_warps=g)
            res[f"batch-{PNAME[prec]}-g{g}"] = host(Ug)
            res[f"batch-{PNAME[prec]}-g{g}-steps"] = steps
            c.close()


def forms_2d(res):
    for (nx, ny) in ((1, 1), (1, 9), (9, 1), (5, 7), (37, 29), (70, 45), (200, 233)):
        for name, bc in (("quadrants", (1, 1, 1, 1)), ("smooth", (0, 0, 0, 0))):
            if name == "quadrants":
                U, dx, dy, _ = I.quadrants_2d(4, nx, ny)
            else:
                U, dx, dy = I.random_smooth_2d(6, nx, ny)
            for prec in (B.T7_F64, B.T7_F32, B.T7_MIXED):
                tag = f"2d-{name}-{nx}x{ny}-{PNAME[prec]}"
                c = B.Context(B.T7_EULER2D, nx, dx, ny=ny, dy=dy, prec=prec, bc=bc, gamma=1.4)
                Ug = torch.tensor(U, dtype=DT[prec], device="cuda")
                L, (mx, my) = c.euler_rhs(Ug, want_masks=True)
                res[tag + "-rhs"], res[tag + "-mx"], res[tag + "-my"] = host(L), mx.cpu().numpy(), my.cpu().numpy()
                c.run(Ug, 0.4, max_steps=3)
                res[tag + "-run"] = host(Ug)
                c.close()


def slabs_2d(res):
    U, dx, dy, _ = I.quadrants_2d(4, 70, 61)
    _, ny, nx = U.shape
    for prec in (B.T7_F64, B.T7_F32, B.T7_MIXED):
        slabs = []
        for r in range(3):
            lo, hi = decomp.partition(ny, 3, r)
            ctx = B.Context(B.T7_EULER2D, nx, dx, ny=hi - lo, dy=dy, prec=prec, bc=(1, 1, 1, 1), gamma=1.4,
                            stream=torch.cuda.Stream())
            slabs.append(decomp.Slab(decomp.CudaSlab(ctx), torch.tensor(U[:, lo:hi], dtype=DT[prec], device="cuda"),
                                     nalpha=2))
        torch.cuda.synchronize()
        comm = decomp.LocalSlabs(slabs, False)
        decomp.rk3_run_slabs(comm, decomp.cfl_dt_2d(dx, dy, 0.4), t_end=math.inf, max_steps=3)
        torch.cuda.synchronize()
        res[f"2d-slabs-{PNAME[prec]}"] = np.concatenate([host(s.state()) for s in slabs], axis=1)


def main(out):
    B.load()
    res = {}
    for part in (forms_1d, adjoint_and_static, slabs_1d, batch, forms_2d, slabs_2d):
        part(res)
    torch.cuda.synchronize()
    np.savez(out, **res)
    print(f"{len(res)} results from {B.LIB_PATH.name}", flush=True)


if __name__ == "__main__":
    main(sys.argv[1])
