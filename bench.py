"""Benchmark of the TENO7-ext hot path: SSP-RK3 steps of the 1D Euler equations
with characteristic-wise TENO7-ext reconstruction on one GB300.

Workload: the Shu-Osher shock / entropy-wave problem (gamma = 1.4; left state
(3.857143, 2.629369, 10.33333) for x < -4, right state (1 + 0.2 sin 5x, 0, 1)
on [-5, 5] with 1600 cells, dx = 1/160), its profile tiled end to end 10486
times to N = 16,777,600 cells (same dx, so the same epsilon = dx^3 and local
structure), zero-gradient ends, CFL 0.5 with the step computed on the device
from max(|u| + c) every step.  A "step" is one full SSP-RK3 step (3 fused stage
launches) over all cells; value = cells x steps / time in Gcell-steps/s.
The state (201 MB in FP32, 403 MB in FP64) is larger than the 129 MB L2, so no
flush is needed between steps.

Lines: the primary line is the FP32 path (dtype f32); the FP64 path (results
bit-identical to the CPU oracle) is reported beside it under "f64", with the
FP32-vs-FP64 error and mask-flip fraction on the 1600-cell Shu-Osher run to
t = 1.8.  `--impl reference` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1808_00037_gb300 import inputs as I  # noqa: E402

TILES = 10486
N1 = 1600
CFL = 0.5
GAMMA = 1.4
# Nominal ALU peaks, for context only: 152 SMs x 128 FP32 lanes x 2 flop per
# FMA x 2.07 GHz, and GB300's nominal FP64 rate.  The roofline divides by the
# rates the library's FMA probe measures on the device (t7_probe_fma).
FP32_NOMINAL_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP64_NOMINAL_TFLOPS = 1.25
# Algorithmic floating-point operations per cell per stage launch of the fused
# 1D-Euler stage kernel (FMA = 2, add/mul/divide/rcp/sqrt/compare = 1), counted
# from the kernel's arithmetic without the warp-tile redundancy and with the
# cutoff evaluated in full:
#   FP32: 31 per-cell staging + 751 per face + 26 update = 808
#   FP64: 30 per-cell staging + 718 per face + 28 update = 776 (no FMA)
FLOPS_PER_CELL_STAGE = {"f32": 808.0, "f64": 776.0}
# Executed floating-point operations per cell per stage launch, from ncu's
# per-opcode thread counters of one launch on the same workload (FMA = 2,
# packed f32x2 FMA = 4, packed add/mul = 2, scalar add/mul = 1; the keep-all
# shortcut skips most of the cutoff, so this is below the algorithmic count);
# None when not captured for the current kernel.
EXEC_FLOPS_PER_CELL_STAGE = {"f32": 584.4, "f64": 812.0}
# DRAM bytes per stage launch per cell measured by ncu (dram__bytes_read.sum +
# dram__bytes_write.sum, averaged over the three stage launches of one RK3
# step at N = 16,777,600) for the current kernels; None when not captured.
TRAFFIC_PER_CELL_LAUNCH = {"f32": 29.50, "f64": None}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup(ngpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reference_arm(args, world, rank):
    """The CPU oracle timed on the host cores (bounded sample of the workload)."""
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    tiles = args.ref_tiles
    U, dx = I.shu_osher(N1, tiles=tiles)
    n = U.shape[1]
    for _ in range(args.warmup):
        U, _, _, _ = oracle.run_1d(oracle.SYS_EULER1D, U, dx, t_end=math.inf, cfl=CFL, bc=(1, 1), max_steps=1)
    t0 = time.perf_counter()
    U, steps, _, _ = oracle.run_1d(oracle.SYS_EULER1D, U, dx, t_end=math.inf, cfl=CFL, bc=(1, 1),
                                   max_steps=args.steps)
    dt = time.perf_counter() - t0
    val = n * steps / dt / 1e9
    line = {
        "impl": "reference", "metric": "TENO7 RK3 Gcell-updates/s (1D Euler, tiled Shu-Osher)", "value": val,
        "unit": "Gcell-steps/s", "n_gpus": world, "steps": steps, "warmup": args.warmup,
        "ms_per_step": dt / steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"Shu-Osher profile (1600 cells on [-5,5], dx=1/160) tiled x{tiles}, "
                               f"N={n} cells (a sample of the x{TILES}, N={N1 * TILES} GPU workload), "
                               f"zero-gradient ends, CFL 0.5, dt from alpha every step",
                   "sample": f"the same profile tiled x{tiles} (N={n}) on the host cores",
                   "parallelism": "host, one thread"},
        "cpu_baseline": {"value": val, "unit": "Gcell-steps/s", "cores": 1, "kind": "oracle",
                         "sample": f"{steps} RK3 steps on {n} cells (single-threaded C oracle)"},
        "e2e": {"value": val, "unit": "Gcell-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _oracle_sample(budget_s, tiles=4):
    """Run the oracle on the tiled Shu-Osher sample for about budget_s seconds;
    returns (cell-steps, seconds).  Also the worker of the all-core run."""
    import oracle
    oracle.build()
    U, dx = I.shu_osher(N1, tiles=tiles)
    n = U.shape[1]
    oracle.run_1d(oracle.SYS_EULER1D, U, dx, t_end=math.inf, cfl=CFL, bc=(1, 1), max_steps=1)
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < budget_s:
        U, s, _, _ = oracle.run_1d(oracle.SYS_EULER1D, U, dx, t_end=math.inf, cfl=CFL, bc=(1, 1), max_steps=10)
        steps += s
    return n * steps, time.perf_counter() - t0


def _oracle_per_form(budget_s=1.5):
    """Single-threaded oracle rates on samples of the other forms' workloads
    (each about budget_s seconds): scalar advection (sin(pi x), 4096 cells),
    2D quadrants (256^2 cells of the 2048^2 recipe) and ragged tubes (the
    first tubes of the 4096-tube batch, their own dx)."""
    import oracle
    oracle.build()
    out = {}
    U, dx, _ = I.advection_sine(4096)
    cells, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        U, s, _, _ = oracle.run_1d(oracle.SYS_ADVECTION, U, dx, t_end=math.inf, cfl=0.2, max_steps=20)
        cells += U.shape[1] * s
    out["advection"] = {"value": cells / (time.perf_counter() - t0) / 1e9, "unit": "Gcell-steps/s",
                        "sample": "sin(pi x), 4096 cells, CFL 0.2"}
    U, dx, dy, _ = I.quadrants_2d(2024, 256, 256)
    cells, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        U, s, _, _ = oracle.run_2d(U, dx, dy, cfl=0.4, max_steps=1)
        cells += 256 * 256 * s
    out["euler2d"] = {"value": cells / (time.perf_counter() - t0) / 1e9, "unit": "Gcell-steps/s",
                      "sample": "four-quadrant data, 256^2 cells"}
    Ub, off, dxs, _ = I.riemann_tube_batch(7, 64)
    cells, t0, t = 0, time.perf_counter(), 0
    while time.perf_counter() - t0 < budget_s and t < 64:
        Ut = Ub[:, off[t]:off[t + 1]]
        _, s, _, _ = oracle.run_1d(oracle.SYS_EULER1D, Ut, dxs[t], t_end=math.inf, cfl=0.5, bc=(1, 1), max_steps=5)
        cells += Ut.shape[1] * s
        t += 1
    out["batch"] = {"value": cells / (time.perf_counter() - t0) / 1e9, "unit": "Gcell-steps/s",
                    "sample": f"5 steps of each of the first {t} tubes of the batch recipe"}
    return out


def cpu_baseline(budget_s=10.0, allcore_s=1.25):
    """The oracle on the host cores: single-threaded for budget_s, then one
    independent copy of the sample per core (processes started with spawn) for
    allcore_s each -- about 30 s of CPU work in all on a 16-core host."""
    import multiprocessing as mp
    cells, dt = _oracle_sample(budget_s)
    one = {"value": cells / dt / 1e9, "unit": "Gcell-steps/s", "cores": 1}
    ncores = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(ncores) as pool:
        t0 = time.perf_counter()
        res = pool.starmap(_oracle_sample, [(allcore_s,)] * ncores)
        wall = time.perf_counter() - t0
    total = sum(r[0] for r in res)
    span = max(r[1] for r in res)
    return {"value": total / span / 1e9, "unit": "Gcell-steps/s", "cores": ncores, "kind": "oracle",
            "sample": f"the Shu-Osher profile tiled x4 (N={N1 * 4}), one independent copy per core, "
                      f"{allcore_s} s each (wall {wall:.1f} s with process start-up)",
            "single_thread": one, "single_thread_other_forms": _oracle_per_form()}


def bench_2d(args, torch, B, dist, world, rank):
    """2D Euler, four-quadrant Riemann data on [0,1]^2 at 2048^2 (seed 2024),
    transmissive boundaries, CFL 0.4: Gcell-steps/s in FP32, mixed precision
    (FP64 state and sums) and FP64."""
    n = 2048
    U0, dx, dy, _ = I.quadrants_2d(2024, n, n)
    out = {"workload": "four-quadrant Riemann data, 2048x2048 on [0,1]^2, transmissive, CFL 0.4"}
    for name, prec, dtype, steps in (("f32", B.T7_F32, torch.float32, args.steps_2d),
                                     ("mixed", B.T7_MIXED, torch.float64, args.steps_2d),
                                     ("f64", B.T7_F64, torch.float64, args.f64_steps_2d)):
        ctx = B.Context(B.T7_EULER2D, n, dx, ny=n, dy=dy, prec=prec, bc=(1, 1, 1, 1), gamma=GAMMA)
        U = torch.tensor(U0, dtype=dtype, device="cuda")
        ctx.run(U, 0.4, max_steps=args.warmup)
        torch.cuda.synchronize()
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        start.record(ctx.stream)
        done, _ = ctx.run(U, 0.4, max_steps=steps)
        end.record(ctx.stream)
        torch.cuda.synchronize()
        ms = start.elapsed_time(end)
        if dist:
            t = torch.tensor([ms], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        assert done == steps
        out[name] = {"value": n * n * steps * world / (ms * 1e-3) / 1e9, "unit": "Gcell-steps/s",
                     "ms_per_step": ms / steps, "steps": steps, "gpu_launches": 6 * steps + 2}
        ctx.close()
        del U
        torch.cuda.empty_cache()
    for name in ("f32", "mixed"):
        out[name]["speedup_vs_f64"] = out["f64"]["ms_per_step"] / out[name]["ms_per_step"]
    return out


def bench_batch(args, torch, B, dist, world, rank):
    """Ragged batch: 4096 Riemann tubes on [0,1], lengths U[256, 8192] (seed 7),
    states rho U[0.1,2], u U[-1,1], p U[0.1,10], each to t = 0.1 at CFL 0.5 in
    one persistent launch.  Gcell-steps/s = sum over tubes of cells x steps /
    time; FP64 and FP32 also timed over a fixed 10 steps of every tube."""
    from oracle import riemann  # exact solution: accuracy check only, not timed
    U0, off, dx, states = I.riemann_tube_batch(7, 4096, 256, 8192)
    out = {"workload": "4096 Riemann tubes per GPU, N ~ U[256, 8192] (17.5M cells), t = 0.1, CFL 0.5"}
    if world > 1:
        # weak scaling: every rank takes its own 4096 tubes (seed 7 + rank), no collective
        U0, off, dx, states = I.riemann_tube_batch(7 + rank, 4096, 256, 8192)
    n = np.diff(off)
    ctx = B.Context(B.T7_EULER1D, U0.shape[1], 1.0, prec=B.T7_F32, bc=(1, 1, 0, 0), gamma=GAMMA)
    U = torch.tensor(U0, dtype=torch.float32, device="cuda")
    g, trial = ctx.batch_autotune(U, off, dx, 0.5, trial_steps=20)
    out["autotune"] = {"group_warps": g, "trial_ms": {str(k): float(v) for k, v in zip((1, 2, 4, 8), trial)}}
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(ctx.stream)
    steps, t = ctx.batch_run(U, off, dx, 0.1, 0.5)
    end.record(ctx.stream)
    torch.cuda.synchronize()
    ms = start.elapsed_time(end)
    cell_steps = float(np.sum(n * steps))
    out["f32"] = {"value": cell_steps * world / (ms * 1e-3) / 1e9, "unit": "Gcell-steps/s", "ms": ms,
                  "cell_steps": cell_steps, "gpu_launches": 2, "all_reached_t_end": bool(np.allclose(t, 0.1))}
    got = U.double().cpu().numpy()
    rng = np.random.default_rng(0)
    errs = []
    for k in rng.choice(4096, 32, replace=False):
        a, b = off[k], off[k + 1]
        x = (np.arange(b - a) + 0.5) / (b - a)
        rho, _, _ = riemann.sample(tuple(states[k, 0]), tuple(states[k, 1]), (x - 0.5) / 0.1)
        errs.append(np.mean(np.abs(got[0, a:b] - rho)) / (np.ptp(rho) + 1e-12))
    out["f32"]["rho_l1_vs_exact_over_range_mean32"] = float(np.mean(errs))
    fixed = {}
    for name, prec, dtype in (("f32", B.T7_F32, torch.float32), ("f64", B.T7_F64, torch.float64)):
        c = B.Context(B.T7_EULER1D, U0.shape[1], 1.0, prec=prec, bc=(1, 1, 0, 0), gamma=GAMMA)
        Ug = torch.tensor(U0, dtype=dtype, device="cuda")
        torch.cuda.synchronize()
        start.record(c.stream)
        st, _ = c.batch_run(Ug, off, dx, 0.1, 0.5, max_steps=10, group_warps=g)
        end.record(c.stream)
        torch.cuda.synchronize()
        fixed[name] = float(np.sum(n * st)) / (start.elapsed_time(end) * 1e-3) / 1e9
        c.close()
    out["fixed_10_steps_gcell_steps_per_s"] = fixed
    out["f32_over_f64"] = fixed["f32"] / fixed["f64"]
    ctx.close()
    return out


def bench_adjoint(args, torch, B):
    """Sine-mode adjoint problem: N = 4096 periodic, 64 modes (seed 11), 2000
    SSP-RK3 steps of fixed dt, checkpoints every 100 steps.  Times a plain
    forward run and the full gradient (checkpointed forward + reverse); the
    reverse cost is reported as a multiple of the forward cost."""
    from paper_1808_00037_gb300 import adjoint as A
    a = I.adjoint_modes(11, K=64)
    out = {"workload": "1D Euler periodic N=4096, 64 sine modes, 2000 RK3 steps, checkpoints every 100"}
    for name, prec in (("f64", B.T7_F64), ("f32", B.T7_F32)):
        J, g, dt = A.sine_modes_gradient(a, n=4096, nsteps=20, every=10, prec=prec)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        A.sine_modes_objective(a, 4096, 2000, dt, prec=prec)
        torch.cuda.synchronize()
        t_fwd = time.perf_counter() - t0
        t0 = time.perf_counter()
        J, g, _ = A.sine_modes_gradient(a, n=4096, nsteps=2000, every=100, prec=prec, dt=dt)
        torch.cuda.synchronize()
        t_grad = time.perf_counter() - t0
        out[name] = {"forward_s": t_fwd, "gradient_s": t_grad,
                     "reverse_over_forward": (t_grad - t_fwd) / t_fwd, "J": J,
                     "grad_norm": float(np.linalg.norm(g))}
    return out


def bench_teno5(args, torch, B, U0, dx, res, dist, world):
    """The TENO5 baseline (Table co1, five-point polynomials selected by each
    face's own cutoff bits) on the same workload and kernels: its throughput
    and the TENO7-ext / TENO5 time ratio per precision -- the measured form of
    the claim that TENO7-ext costs about as much as TENO5."""
    n = U0.shape[1]
    out = {"workload": "same tiled Shu-Osher state and step count as the TENO7-ext lines"}
    for name, prec, dtype in (("f32", B.T7_F32, torch.float32), ("f64", B.T7_F64, torch.float64)):
        if name not in res:
            continue
        steps = res[name]["steps"]
        ctx = B.Context(B.T7_EULER1D, n, dx, prec=prec, bc=(1, 1, 0, 0), gamma=GAMMA, scheme=B.T7_TENO5)
        U = torch.tensor(U0, dtype=dtype, device="cuda")
        ctx.run(U, CFL, max_steps=args.warmup)
        torch.cuda.synchronize()
        ms, _ = time_run(torch, ctx, U, steps, dist, world)
        out[name] = {"value": n * steps * world / (ms * 1e-3) / 1e9, "unit": "Gcell-steps/s",
                     "ms_per_step": ms / steps, "steps": steps,
                     "teno7ext_over_teno5_time": res[name]["ms_per_step"] / (ms / steps)}
        ctx.close()
        del U
        torch.cuda.empty_cache()
    return out


def bench_alpha_mode(args, torch, B, U0, dx, res, dist, world):
    """The per-field Lax-Friedrichs alpha (t7_grid.alpha_mode = per field:
    alpha_k = max |lambda_k| per characteristic field, splits formed from
    the projections of F and U) on the same workload in FP32: its throughput
    and its time against the global alpha's."""
    n = U0.shape[1]
    steps = args.steps
    ctx = B.Context(B.T7_EULER1D, n, dx, prec=B.T7_F32, bc=(1, 1, 0, 0), gamma=GAMMA,
                    alpha_mode=B.T7_ALPHA_PER_FIELD)
    U = torch.tensor(U0, dtype=torch.float32, device="cuda")
    ctx.run(U, CFL, max_steps=args.warmup)
    torch.cuda.synchronize()
    ms, _ = time_run(torch, ctx, U, steps, dist, world)
    out = {"workload": "same tiled Shu-Osher state and step count as the primary line, FP32",
           "value": n * steps * world / (ms * 1e-3) / 1e9, "unit": "Gcell-steps/s", "ms_per_step": ms / steps,
           "steps": steps}
    if "f32" in res:
        out["time_vs_global_alpha"] = (ms / steps) / res["f32"]["ms_per_step"]
    ctx.close()
    del U
    torch.cuda.empty_cache()
    return out


def bench_mixed(args, torch, B, U0, dx, res, dist, world):
    """Mixed precision (FP64 state, FP32 reconstruction, FP64 flux difference
    and RK combination) on the same workload: throughput, its speedup over the
    FP64 path, and the drift of the domain sums over the timed steps with
    periodic ends (FP64 round-off, against the FP32 state's)."""
    n = U0.shape[1]
    steps = args.steps
    ctx = B.Context(B.T7_EULER1D, n, dx, prec=B.T7_MIXED, bc=(1, 1, 0, 0), gamma=GAMMA)
    U = torch.tensor(U0, dtype=torch.float64, device="cuda")
    ctx.run(U, CFL, max_steps=args.warmup)
    torch.cuda.synchronize()
    ms, _ = time_run(torch, ctx, U, steps, dist, world)
    out = {"value": n * steps * world / (ms * 1e-3) / 1e9, "unit": "Gcell-steps/s", "ms_per_step": ms / steps,
           "steps": steps, "gpu_launches": 3 * steps + 2}
    if "f64" in res:
        out["speedup_vs_f64"] = res["f64"]["ms_per_step"] / (ms / steps)
    if "f32" in res:
        out["time_vs_f32"] = (ms / steps) / res["f32"]["ms_per_step"]
    ctx.close()
    drift = {}
    for name, prec, dtype in (("mixed", B.T7_MIXED, torch.float64), ("f32", B.T7_F32, torch.float32)):
        c = B.Context(B.T7_EULER1D, n, dx, prec=prec, bc=(0, 0, 0, 0), gamma=GAMMA)
        Ug = torch.tensor(U0, dtype=dtype, device="cuda")
        s0 = Ug.double().sum(dim=1)
        c.run(Ug, CFL, max_steps=steps)
        s1 = Ug.double().sum(dim=1)
        drift[name] = float(((s1 - s0).abs() / Ug.double().abs().sum(dim=1)).max().item())
        c.close()
        del Ug
    out["periodic_sum_drift"] = {**drift, "steps": steps}
    del U
    torch.cuda.empty_cache()
    return out


def bench_advection(args, torch, B, dist, world):
    """Scalar advection u_t + u_x = 0, sin(pi x) on [-1, 1], periodic, N = 2^24
    cells, CFL 0.2 (the advection configuration's data at a timed size): the
    lightest system (m = 1), for its HBM fraction -- 8 m s bytes per
    cell-step, one stage reads U (and U^n) and writes the stage state."""
    n = 1 << 24
    U0, dx, _ = I.advection_sine(n)
    hbm_peak, peak_kind = peaks()
    out = {"workload": f"advection sin(pi x) on [-1,1], N={n}, periodic, CFL 0.2"}
    # FP32: a step takes ~0.25 ms, so 100 timed steps after 10 warm-up steps
    # (a 20-step region right after the upload read ~15% low: the device had
    # not settled)
    for name, prec, dtype, steps, warm in (("f32", B.T7_F32, torch.float32, max(args.steps, 100), max(args.warmup, 10)),
                                           ("f64", B.T7_F64, torch.float64, max(2, args.steps // 10), args.warmup)):
        ctx = B.Context(B.T7_SCALAR_ADVECTION, n, dx, prec=prec, bc=(0, 0, 0, 0), adv_speed=1.0)
        U = torch.tensor(U0, dtype=dtype, device="cuda")
        ctx.run(U, 0.2, max_steps=warm)
        torch.cuda.synchronize()
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        start.record(ctx.stream)
        done, _ = ctx.run(U, 0.2, max_steps=steps)
        end.record(ctx.stream)
        torch.cuda.synchronize()
        ms = start.elapsed_time(end)
        assert done == steps
        s_ = 4 if name == "f32" else 8
        gbs = 8 * s_ * n * steps / (ms * 1e-3) / 1e9
        out[name] = {"value": n * steps * world / (ms * 1e-3) / 1e9, "unit": "Gcell-steps/s",
                     "ms_per_step": ms / steps, "steps": steps,
                     "hbm": {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                             "peak_kind": peak_kind, "bytes_per_cell_step": 8 * s_}}
        ctx.close()
        del U
        torch.cuda.empty_cache()
    return out


def alu_peaks(B):
    """FP32 and FP64 FMA rates measured on this device by the library's probe
    (t7_probe_fma: every SM full of independent FMA chains); the FP32
    denominator is the faster of the scalar and the packed f32x2 form."""
    f32, _ = B.probe_fma(B.T7_PROBE_F32, iters=2048, repeats=5)
    f32x2, _ = B.probe_fma(B.T7_PROBE_F32X2, iters=2048, repeats=5)
    f64, _ = B.probe_fma(B.T7_PROBE_F64, iters=256, repeats=5)
    return {"f32": max(f32, f32x2), "f64": f64, "f32_scalar": f32, "f32x2": f32x2,
            "kind": "measured: t7_probe_fma FMA-chain probe (f32: max of scalar and f32x2)"}


def _rel_l1(a, b):
    return float((a.double() - b.double()).abs().sum() / b.double().abs().sum())


def _flips(ma, mb):
    if isinstance(ma, tuple):
        d = sum(int((x != y).sum()) for x, y in zip(ma, mb))
        return d / sum(x.numel() for x in ma)
    return float((ma != mb).double().mean())


def _trajectory(torch, B, make, U0, cfl, t_end, nchk, lo_prec):
    """The same problem run in FP64 and in lo_prec (FP32 or mixed) side by
    side to t_end in nchk equal chunks.  At each chunk end: the fraction of
    Delta masks that differ with each precision evaluating its own state
    (trajectory), and with the low precision evaluating the FP64 state (same
    state); at the end the relative L1 error of every variable against FP64."""
    c64, clo = make(B.T7_F64), make(lo_prec)
    lo_dtype = torch.float32 if lo_prec == B.T7_F32 else torch.float64
    U64 = torch.tensor(U0, dtype=torch.float64, device="cuda")
    Ulo = torch.tensor(U0, dtype=lo_dtype, device="cuda")
    traj, same = [], []
    for k in range(nchk):
        c64.run(U64, cfl, t_end=t_end / nchk)
        clo.run(Ulo, cfl, t_end=t_end / nchk)
        m64 = c64.euler_rhs(U64, want_masks=True)[1]
        traj.append(_flips(m64, clo.euler_rhs(Ulo, want_masks=True)[1]))
        same.append(_flips(m64, clo.euler_rhs(U64.to(lo_dtype), want_masks=True)[1]))
    out = {"rel_l1_vs_f64": _rel_l1(Ulo, U64), "mask_flip_trajectory": traj, "mask_flip_same_state": same,
           "checkpoints": nchk}
    c64.close()
    clo.close()
    return out


def bench_accuracy(args, torch, B):
    """Accuracy of the reduced-precision forms against the FP64 path on the
    configurations' smooth and shock cases: relative L1 error (the smooth
    gate is 1e-5) and mask-flip fractions along the trajectory."""
    out = {}
    Us, dxs, _ = I.random_euler_smooth(9, N1)
    Ua, dxa = I.shu_osher(N1)

    def mk1(U, dx, bc):
        return lambda prec: B.Context(B.T7_EULER1D, U.shape[1], dx, prec=prec, bc=bc, gamma=GAMMA)
    for form, prec in (("f32", B.T7_F32), ("mixed", B.T7_MIXED)):
        out[f"euler1d_{form}"] = {
            "smooth": {"case": f"random smooth periodic Euler, N={N1}, t=0.25",
                       **_trajectory(torch, B, mk1(Us, dxs, (0, 0, 0, 0)), Us, CFL, 0.25, 5, prec)},
            "shock": {"case": f"Shu-Osher N={N1}, t=1.8",
                      **_trajectory(torch, B, mk1(Ua, dxa, (1, 1, 0, 0)), Ua, CFL, 1.8, 6, prec)}}
    n2 = 256
    U2s, dx2s, dy2s = I.random_smooth_2d(4, n2, n2)
    U2q, dx2q, dy2q, _ = I.quadrants_2d(2024, n2, n2)

    def mk2(dx, dy, bc):
        return lambda prec: B.Context(B.T7_EULER2D, n2, dx, ny=n2, dy=dy, prec=prec, bc=bc, gamma=GAMMA)
    for form, prec in (("f32", B.T7_F32), ("mixed", B.T7_MIXED)):
        out[f"euler2d_{form}"] = {
            "smooth": {"case": f"random smooth periodic 2D Euler, {n2}^2, t=0.05",
                       **_trajectory(torch, B, mk2(dx2s, dy2s, (0, 0, 0, 0)), U2s, 0.4, 0.05, 4, prec)},
            "shock": {"case": f"four-quadrant Riemann data, {n2}^2, t=0.1",
                      **_trajectory(torch, B, mk2(dx2q, dy2q, (1, 1, 1, 1)), U2q, 0.4, 0.1, 4, prec)}}
    # ragged batch: the first 32 tubes of the batch recipe to t = 0.1 in FP32 and FP64
    Ub, off, dxb, _ = I.riemann_tube_batch(7, 32, 256, 8192)
    res = {}
    for name, prec, dtype in (("f32", B.T7_F32, torch.float32), ("f64", B.T7_F64, torch.float64)):
        c = B.Context(B.T7_EULER1D, Ub.shape[1], 1.0, prec=prec, bc=(1, 1, 0, 0), gamma=GAMMA)
        Ug = torch.tensor(Ub, dtype=dtype, device="cuda")
        c.batch_run(Ug, off, dxb, 0.1, 0.5)
        res[name] = Ug
        c.close()
    flips = []
    for t in range(0, 32, 4):
        a, b = off[t], off[t + 1]
        cs = [B.Context(B.T7_EULER1D, b - a, dxb[t], prec=p, bc=(1, 1, 0, 0), gamma=GAMMA)
              for p in (B.T7_F64, B.T7_F32)]
        m64 = cs[0].euler_rhs(res["f64"][:, a:b].contiguous(), want_masks=True)[1]
        m32 = cs[1].euler_rhs(res["f32"][:, a:b].contiguous(), want_masks=True)[1]
        flips.append(_flips(m64, m32))
        for c in cs:
            c.close()
    out["batch_f32"] = {"case": "first 32 tubes of the 4096-tube recipe (seed 7), t=0.1",
                        "rel_l1_vs_f64": _rel_l1(res["f32"], res["f64"]),
                        "mask_flip_end_state": float(np.mean(flips)), "tubes_for_masks": 8}
    gate = 1e-5
    out["smooth_gate"] = {"limit": gate, "pass": all(
        out[k]["smooth"]["rel_l1_vs_f64"] <= gate for k in out if "smooth" in out[k])}
    return out


def bench_strong(args, torch, B, U0, dx, dist, world, rank):
    """Strong scaling: one domain split into `world` slabs, one per rank, each
    advanced by the CUDA slab stages with 4-cell (row) halos exchanged by NCCL
    point-to-point messages and the alphas of every stage all-reduced (max)
    on the device (paper_1808_00037_gb300.decomp): the 16.8M-cell tiled
    Shu-Osher domain (1D) and the 2048^2 quadrant domain (2D, split along y).
    FP32, CFL steps as in the primary lines."""
    from paper_1808_00037_gb300 import decomp
    U2, dx2, dy2, _ = I.quadrants_2d(2024, 2048, 2048)
    out = {"scaling": "strong",
           "timing": "host wall clock between barriers and device synchronisations (max over ranks)",
           "parallelism": f"slab decomposition over {world} ranks, NCCL halos + all-reduce(max) of alpha"}
    for name, U, sysid, dt_of, nalpha in (("euler1d", U0, B.T7_EULER1D, decomp.cfl_dt_1d(dx, CFL), 1),
                                          ("euler2d", U2, B.T7_EULER2D, decomp.cfl_dt_2d(dx2, dy2, 0.4), 2)):
        lo, hi = decomp.partition(U.shape[1], world, rank)
        if sysid == B.T7_EULER2D:
            ctx = B.Context(sysid, U.shape[2], dx2, ny=hi - lo, dy=dy2, prec=B.T7_F32, bc=(1, 1, 1, 1), gamma=GAMMA)
        else:
            ctx = B.Context(sysid, hi - lo, dx, prec=B.T7_F32, gamma=GAMMA)
        slab = decomp.Slab(decomp.CudaSlab(ctx), torch.tensor(U[:, lo:hi], dtype=torch.float32, device="cuda"),
                           nalpha=nalpha)
        comm = decomp.RankSlabs(slab, periodic=False)
        decomp.rk3_run_slabs(comm, dt_of, t_end=math.inf, max_steps=args.warmup)
        torch.cuda.synchronize()
        dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        steps, _ = decomp.rk3_run_slabs(comm, dt_of, t_end=math.inf, max_steps=args.steps)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        t = torch.tensor([el], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        el = float(t.item())
        ctx.close()
        cells = U[0].size
        out[name] = {"value": cells * steps / el / 1e9, "unit": "Gcell-steps/s", "ms_per_step": el / steps * 1e3,
                     "steps": steps, "cells_total": int(cells)}
    return out


def bench_slabs_local(args, torch, B, U1, dx1, nslabs=2):
    """The slab decomposition on one GPU: the 16.8M-cell tiled Shu-Osher
    domain (1D) and the 2048^2 quadrant domain (2D, cut along y) in `nslabs`
    slabs, each with its own context and CUDA stream, 4-cell (row) halos
    filled by device-local copies and the alphas of every stage all-reduced
    (a max over the slabs) on the device (paper_1808_00037_gb300.decomp).
    FP32.  The rate beside the unsplit kernels' is the cost of the
    decomposition machinery itself (halo copies, per-stage reductions, one
    host read of dt per step).  Host wall clock between device
    synchronisations."""
    from paper_1808_00037_gb300 import decomp
    out = {"workload": f"{nslabs} slabs on {nslabs} CUDA streams of one GPU, FP32",
           "timing": "host wall clock between device synchronisations"}
    U2, dx2, dy2, _ = I.quadrants_2d(2024, 2048, 2048)
    cases = (("euler1d", U1, B.T7_EULER1D, decomp.cfl_dt_1d(dx1, CFL), 1),
             ("euler2d", U2, B.T7_EULER2D, decomp.cfl_dt_2d(dx2, dy2, 0.4), 2))
    for name, U, sysid, dt_of, nalpha in cases:
        rows = U.shape[1]
        slabs = []
        for r in range(nslabs):
            lo, hi = decomp.partition(rows, nslabs, r)
            st = torch.cuda.Stream()
            if sysid == B.T7_EULER2D:
                ctx = B.Context(sysid, U.shape[2], dx2, ny=hi - lo, dy=dy2, prec=B.T7_F32, bc=(1, 1, 1, 1),
                                gamma=GAMMA, stream=st)
            else:
                ctx = B.Context(sysid, hi - lo, dx1, prec=B.T7_F32, bc=(1, 1, 0, 0), gamma=GAMMA, stream=st)
            Ul = torch.tensor(U[:, lo:hi], dtype=torch.float32, device="cuda")
            slabs.append(decomp.Slab(decomp.CudaSlab(ctx), Ul, nalpha=nalpha))
        comm = decomp.LocalSlabs(slabs, periodic=False)
        decomp.rk3_run_slabs(comm, dt_of, t_end=math.inf, max_steps=args.warmup)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        steps, _ = decomp.rk3_run_slabs(comm, dt_of, t_end=math.inf, max_steps=args.steps)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        cells = U[0].size
        out[name] = {"value": cells * steps / el / 1e9, "unit": "Gcell-steps/s", "ms_per_step": el / steps * 1e3,
                     "steps": steps, "cells": int(cells)}
        for sl in slabs:
            sl.backend.ctx.close()
        del slabs, comm
        torch.cuda.empty_cache()
    return out


def time_run(torch, ctx, U, steps, dist, world, sampler_index=None):
    stream = ctx.stream
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(sampler_index) if sampler_index is not None else None
    if sampler:
        sampler.__enter__()
    start.record(stream)
    done, _ = ctx.run(U, CFL, max_steps=steps)
    end.record(stream)
    torch.cuda.synchronize()
    if sampler:
        sampler.__exit__()
    ms = start.elapsed_time(end)
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        dist.barrier()
    assert done == steps
    return ms, (sampler.summary() if sampler else None)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tiles", type=int, default=TILES)
    ap.add_argument("--ref-tiles", type=int, default=64)
    ap.add_argument("--f64-steps", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-2d", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-teno5", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-advection", action="store_true")
    ap.add_argument("--no-strong", action="store_true")
    ap.add_argument("--steps-2d", type=int, default=20)
    ap.add_argument("--f64-steps-2d", type=int, default=3)
    ap.add_argument("--only", choices=["f32", "f64", "2d", "batch", "adjoint", "advection", "slabs"], default=None,
                    help="time one 1D precision, or only the 2D case (profiling)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # one process per GPU: re-run this command under torchrun
        import socket
        sock = socket.socket()
        sock.bind(("127.0.0.1", 0))
        port = sock.getsockname()[1]
        sock.close()
        cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", str(args.gpus),
               "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__)] + sys.argv[1:]
        return subprocess.call(cmd)
    world, rank, local = dist_setup(args.gpus)

    if args.impl == "reference":
        return reference_arm(args, world, rank)

    import torch
    from paper_1808_00037_gb300 import binding as B

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist_mod.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist = dist_mod

    if args.only == "adjoint":
        if rank == 0:
            print(json.dumps({"only": "adjoint", **bench_adjoint(args, torch, B)}), flush=True)
        return 0
    if args.only == "advection":
        if rank == 0:
            print(json.dumps({"only": "advection", **bench_advection(args, torch, B, dist, world)}), flush=True)
        return 0
    if args.only in ("2d", "batch"):
        r2 = (bench_2d if args.only == "2d" else bench_batch)(args, torch, B, dist, world, rank)
        if rank == 0:
            print(json.dumps({"only": args.only, **r2}), flush=True)
        return 0
    U0, dx = I.shu_osher(N1, tiles=args.tiles)
    n = U0.shape[1]
    if args.only == "slabs":
        if rank == 0:
            print(json.dumps({"only": "slabs", **bench_slabs_local(args, torch, B, U0, dx)}), flush=True)
        return 0
    hbm_peak, peak_kind = peaks()
    alu = alu_peaks(B)
    res = {}
    for name, prec, dtype in (("f32", B.T7_F32, torch.float32), ("f64", B.T7_F64, torch.float64)):
        if args.only and name != args.only:
            continue
        steps = args.steps if name == "f32" or args.f64_steps is None else args.f64_steps
        ctx = B.Context(B.T7_EULER1D, n, dx, prec=prec, bc=(1, 1, 0, 0), gamma=GAMMA)
        U = torch.tensor(U0, dtype=dtype, device="cuda")
        ctx.run(U, CFL, max_steps=args.warmup)
        torch.cuda.synchronize()
        ms, clocks = time_run(torch, ctx, U, steps, dist, world, sampler_index=local if rank == 0 else None)
        s = 4 if name == "f32" else 8
        launches = 3 * steps
        # the fused stage kernel is the only per-step launch (2 small launches
        # per run set up the control block and alpha): its average duration is
        # the timed region over the stage launches
        stage_ms = ms / launches
        alg_bytes = 8 * 3 * s / 3 * n  # per stage launch, averaged over the three stages
        achieved = alg_bytes / (stage_ms * 1e-3) / 1e9
        flops = FLOPS_PER_CELL_STAGE[name] * n
        tflops = flops / (stage_ms * 1e-3) / 1e12
        peak_alu = alu[name]
        tr = TRAFFIC_PER_CELL_LAUNCH[name]
        ex = EXEC_FLOPS_PER_CELL_STAGE[name]
        ex_tflops = None if ex is None else ex * n / (stage_ms * 1e-3) / 1e12
        res[name] = {
            "value": n * steps * world / (ms * 1e-3) / 1e9, "ms_per_step": ms / steps, "steps": steps,
            "clocks": clocks, "gpu_launches": launches + 2, "stage_launch_ms": stage_ms,
            "roofline": {"bound": "alu", "achieved": tflops, "peak": peak_alu, "unit": "TFLOP/s",
                         "frac": tflops / peak_alu, "traffic": None if tr is None else tr * n,
                         "flops_per_cell_stage": FLOPS_PER_CELL_STAGE[name],
                         "flops_kind": "algorithmic (cutoff counted in full)",
                         "executed": {"flops_per_cell_stage": ex, "achieved": ex_tflops,
                                      "frac": None if ex is None else ex_tflops / peak_alu},
                         "peak_kind": alu["kind"],
                         "nominal_peak": FP32_NOMINAL_TFLOPS if name == "f32" else FP64_NOMINAL_TFLOPS},
            "hbm": {"achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                    "peak_kind": peak_kind, "bytes_per_cell_step": 8 * 3 * s,
                    "traffic": None if tr is None else tr * n},
        }
        # end-to-end through the host-array entry point: per step H2D + step + D2H
        if not args.no_e2e:
            Uh = torch.tensor(U0, dtype=dtype).pin_memory()
            ctx.run_host(Uh, CFL, max_steps=1)
            e2e_steps = min(steps, 10)
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(e2e_steps):
                ctx.run_host(Uh, CFL, max_steps=1)
            el = time.perf_counter() - t0
            if dist:
                t = torch.tensor([el], device="cuda")
                dist.all_reduce(t, op=dist.ReduceOp.MAX)
                el = float(t.item())
            nbytes = U0.size * s
            res[name]["e2e"] = {"value": n * e2e_steps * world / el / 1e9, "unit": "Gcell-steps/s",
                                "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes}
        ctx.close()
        del U
        torch.cuda.empty_cache()

    if args.only:
        if rank == 0:
            print(json.dumps({"only": args.only, **res[args.only]}), flush=True)
        return 0
    res5 = None if args.no_teno5 else bench_teno5(args, torch, B, U0, dx, res, dist, world)
    resm = None if args.no_mixed else bench_mixed(args, torch, B, U0, dx, res, dist, world)
    resp = None if args.no_mixed else bench_alpha_mode(args, torch, B, U0, dx, res, dist, world)
    resv = None if args.no_advection else bench_advection(args, torch, B, dist, world)
    res2d = None if args.no_2d else bench_2d(args, torch, B, dist, world, rank)
    resb = None if args.no_batch else bench_batch(args, torch, B, dist, world, rank)
    resa = None if (args.no_adjoint or rank != 0) else bench_adjoint(args, torch, B)
    # accuracy at the quoted configuration: 1600 cells to t = 1.8, FP32 vs FP64
    # accuracy of the FP32 and mixed forms against FP64 (smooth and shock
    # cases of every form), on rank 0
    acc = None if (args.no_accuracy or rank != 0) else bench_accuracy(args, torch, B)
    strong = None if (world == 1 or args.no_strong) else bench_strong(args, torch, B, U0, dx, dist, world, rank)
    slabs1 = None if (world > 1 or args.no_strong) else bench_slabs_local(args, torch, B, U0, dx)
    if slabs1:
        slabs1["euler1d"]["vs_unsplit"] = slabs1["euler1d"]["value"] / res["f32"]["value"]
        if res2d:
            slabs1["euler2d"]["vs_unsplit"] = slabs1["euler2d"]["value"] / res2d["f32"]["value"]

    if rank != 0:
        return 0
    # the oracle on the host cores: on rank 0 of a one-GPU run only
    cpu = None if (args.no_cpu_baseline or world > 1) else cpu_baseline()
    main_res = res["f32"]
    line = {
        "metric": "TENO7 RK3 Gcell-updates/s (1D Euler, tiled Shu-Osher)", "value": main_res["value"],
        "unit": "Gcell-steps/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": main_res["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"Shu-Osher profile (1600 cells on [-5,5], dx=1/160) tiled x{args.tiles}, "
                               f"N={n} cells per GPU, zero-gradient ends, CFL 0.5, device-side dt",
                   "l2": "inputs larger than L2 (state 201 MB f32 / 403 MB f64 > 129 MB)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": main_res["roofline"],
        "hbm_roofline": main_res["hbm"],
        "clocks": main_res["clocks"], "gpu_launches": main_res["gpu_launches"],
        "e2e": main_res.get("e2e"),
        "f64": res["f64"], "mixed": resm, "teno5": res5, "advection": resv, "accuracy": acc, "euler2d": res2d,
        "batch": resb, "adjoint": resa, "strong": strong, "slabs_1gpu": slabs1, "per_field_alpha": resp,
        "alu_peaks": alu,
        "cpu_baseline": cpu,
    }
    # compact FP64 figures at the end of the line, where a reader of its tail finds them
    f64r = res.get("f64")
    if f64r:
        line["f64_summary"] = {"value": f64r["value"], "unit": "Gcell-steps/s", "ms_per_step": f64r["ms_per_step"],
                               "steps": f64r["steps"], "f32_over_f64": main_res["value"] / f64r["value"]}
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
