"""Thin Python binding of libteno7 (include/teno7.h): argument marshalling only.

Every step of the scheme runs in the CUDA kernels behind the C ABI; this module
loads the in-tree shared library with ctypes, allocates output tensors with
PyTorch (device memory and streams only) and passes raw pointers.  There is no
CPU fallback: if the library is missing, loading fails with an error.
"""
from __future__ import annotations

import ctypes
import math
import os
from pathlib import Path

import numpy as np

PKG = Path(__file__).resolve().parent
# the release build; T7_LIBRARY names another build of the same library (the
# index-checked libteno7_checked.so)
LIB_PATH = Path(os.environ["T7_LIBRARY"]) if os.environ.get("T7_LIBRARY") else PKG / "libteno7.so"

T7_OK, T7_EINVAL, T7_ECUDA, T7_ENONPHYSICAL, T7_ENONFINITE, T7_ETIMEOUT, T7_ENOMEM = 0, -1, -2, -3, -4, -5, -6
T7_EINDEX = -7
T7_BC_PERIODIC, T7_BC_ZERO_GRADIENT = 0, 1
T7_F64, T7_F32, T7_MIXED = 0, 1, 2
T7_SCALAR_ADVECTION, T7_EULER1D, T7_EULER2D, T7_BURGERS = 0, 1, 2, 3
T7_TENO7EXT, T7_TENO5 = 0, 1
T7_ALPHA_GLOBAL, T7_ALPHA_PER_FIELD = 0, 1
T7_PROBE_F32, T7_PROBE_F32X2, T7_PROBE_F64 = 0, 1, 2

_STATUS = {0: "T7_OK", -1: "T7_EINVAL", -2: "T7_ECUDA", -3: "T7_ENONPHYSICAL", -4: "T7_ENONFINITE",
           -5: "T7_ETIMEOUT", -6: "T7_ENOMEM", -7: "T7_EINDEX"}


class T7Error(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class t7_grid(ctypes.Structure):
    _fields_ = [("sys", ctypes.c_int), ("prec", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("bc", ctypes.c_int * 4),
                ("gamma", ctypes.c_double), ("adv_speed", ctypes.c_double), ("CT", ctypes.c_double),
                ("eps_x", ctypes.c_double), ("eps_y", ctypes.c_double), ("scheme", ctypes.c_int),
                ("alpha_mode", ctypes.c_int)]


_lib = None


def load(path: Path | str | None = None) -> ctypes.CDLL:
    """Load libteno7.so (build it first with __graft_entry__.build() or
    paper_1808_00037_gb300.build.build())."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = Path(path) if path else LIB_PATH
    if not p.exists():
        raise RuntimeError(f"CUDA library {p} is missing: build it first (no CPU fallback exists)")
    lib = ctypes.CDLL(str(p))
    vp, i, d, u8p = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    sigs = {
        "t7_create": ([ctypes.POINTER(t7_grid), vp, ctypes.POINTER(vp)], i),
        "t7_destroy": ([vp], i),
        "t7_set_stream": ([vp, vp], i),
        "t7_last_error": ([vp], ctypes.c_char_p),
        "t7_sync": ([vp], i),
        "t7_teno7_reconstruct": ([vp, vp, i, i, d, vp, u8p, u8p], i),
        "t7_euler_rhs": ([vp, vp, vp, u8p], i),
        "t7_cfl_dt": ([vp, vp, d, ctypes.POINTER(d)], i),
        "t7_rk3_step": ([vp, vp, d], i),
        "t7_run": ([vp, vp, d, d, i, ctypes.POINTER(i), ctypes.POINTER(d)], i),
        "t7_run_host": ([vp, vp, d, d, i, ctypes.POINTER(i), ctypes.POINTER(d)], i),
        "t7_rk3_step_static": ([ctypes.POINTER(t7_grid), vp, d, vp, ctypes.c_char_p, ctypes.c_size_t], i),
        "t7_batch_run": ([vp, vp, vp, vp, i, d, d, i, i, vp, vp], i),
        "t7_euler_rhs_adjoint": ([vp, vp, vp, vp], i),
        "t7_rk3_step_adjoint": ([vp, vp, d, vp], i),
        "t7_tape_bytes": ([vp, ctypes.POINTER(ctypes.c_size_t)], i),
        "t7_rk3_step_record": ([vp, vp, vp, d, vp], i),
        "t7_rk3_step_adjoint_recorded": ([vp, vp, vp, d, vp], i),
        "t7_batch_autotune": ([vp, vp, vp, vp, i, d, i, ctypes.POINTER(i), vp], i),
        "t7_probe_fma": ([i, i, i, vp, ctypes.POINTER(d), ctypes.POINTER(ctypes.c_float)], i),
        "t7_probe_index_check": ([i, i, i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)], i),
        "t7_slab_alpha": ([vp, vp, vp], i),
        "t7_slab_rhs": ([vp, vp, vp, vp, u8p], i),
        "t7_slab_stage": ([vp, i, vp, vp, vp, vp, d, vp], i),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    if path is None:
        _lib = lib
    return lib


def _ptr(t) -> int | None:
    if t is None:
        return None
    return t.data_ptr()


class Context:
    """One problem (grid + parameters + precision) bound to a CUDA stream."""

    def __init__(self, sys: int, nx: int, dx: float, *, prec: int = T7_F64, ny: int = 1, dy: float = 0.0,
                 bc=(T7_BC_PERIODIC,) * 4, gamma: float = 1.4, adv_speed: float = 1.0, CT: float = 1e-5,
                 eps_x: float = -1.0, eps_y: float = -1.0, scheme: int = 0, alpha_mode: int = 0, stream=None):
        import torch
        self._torch = torch
        self.lib = load()
        self.sys, self.prec, self.nx, self.ny = sys, prec, nx, ny
        self.m = {T7_SCALAR_ADVECTION: 1, T7_BURGERS: 1, T7_EULER1D: 3, T7_EULER2D: 4}[sys]
        self.dtype = torch.float32 if prec == T7_F32 else torch.float64  # mixed: FP64 state
        self.np_dtype = np.float32 if prec == T7_F32 else np.float64
        bc = tuple(bc) + (T7_BC_PERIODIC,) * (4 - len(bc))
        g = t7_grid(sys, prec, nx, ny, dx, dy, (ctypes.c_int * 4)(*bc), gamma, adv_speed, CT, eps_x, eps_y, scheme,
                    alpha_mode)
        self.scheme = scheme
        self.grid = g
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        st = self.lib.t7_create(ctypes.byref(g), ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h))
        if st != T7_OK:
            raise T7Error(st, "t7_create failed")
        self.h = h

    def set_stream(self, stream):
        """Run later calls on `stream` (a torch.cuda.Stream); work queued on the
        previous stream is ordered before them."""
        self._check(self.lib.t7_set_stream(self.h, ctypes.c_void_p(stream.cuda_stream)), "t7_set_stream")
        self.stream = stream

    def close(self):
        if getattr(self, "h", None):
            self.lib.t7_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int, what: str):
        if st != T7_OK:
            raise T7Error(st, f"{what}: {self.lib.t7_last_error(self.h).decode()}")

    def _dev(self, t):
        torch = self._torch
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == self.dtype and t.is_contiguous()):
            raise ValueError(f"expected a contiguous CUDA tensor of dtype {self.dtype}")
        return t

    # ------------------------------------------------------------ the ABI --
    def teno7_reconstruct(self, v_padded, sign: int, eps: float, want_bits: bool = False):
        torch = self._torch
        v = self._dev(v_padded)
        n = v.numel() - 8
        fhat = torch.empty(n + 1, dtype=self.dtype, device=v.device)
        d3 = torch.empty(n + 3, dtype=torch.uint8, device=v.device) if want_bits else None
        D5 = torch.empty(n + 1, dtype=torch.uint8, device=v.device) if want_bits else None
        self._check(self.lib.t7_teno7_reconstruct(self.h, _ptr(v), n, sign, eps, _ptr(fhat), _ptr(d3), _ptr(D5)),
                    "t7_teno7_reconstruct")
        return fhat, d3, D5

    def euler_rhs(self, U, want_masks: bool = False, out=None):
        """L(U).  masks: 1D [2, m, nx+1]; 2D a pair (x faces [2, 4, ny, nx+1],
        y faces [2, 4, nx, ny+1])."""
        torch = self._torch
        U = self._dev(U)
        out = torch.empty_like(U) if out is None else self._dev(out)
        masks = None
        if want_masks:
            if self.sys == T7_EULER2D:
                nx, ny = self.nx, self.ny
                masks = torch.empty(8 * ny * (nx + 1) + 8 * nx * (ny + 1), dtype=torch.uint8, device=U.device)
            else:
                masks = torch.empty((2, self.m, self.nx + 1), dtype=torch.uint8, device=U.device)
        self._check(self.lib.t7_euler_rhs(self.h, _ptr(U), _ptr(out), _ptr(masks)), "t7_euler_rhs")
        if want_masks and self.sys == T7_EULER2D:
            k = 8 * self.ny * (self.nx + 1)
            masks = (masks[:k].view(2, 4, self.ny, self.nx + 1), masks[k:].view(2, 4, self.nx, self.ny + 1))
        return out, masks

    def cfl_dt(self, U, cfl: float) -> float:
        dt = ctypes.c_double()
        self._check(self.lib.t7_cfl_dt(self.h, _ptr(self._dev(U)), cfl, ctypes.byref(dt)), "t7_cfl_dt")
        return dt.value

    # -- slabs of a decomposed domain: padded arrays [m, nx + 8] (2D [4, ny + 8, nx]), device alphas
    def _padded(self, t):
        t = self._dev(t)
        if self.sys == T7_EULER2D:
            shape = (4, self.ny + 8, self.nx)
            if tuple(t.shape) != shape:
                raise ValueError(f"expected a padded slab array {list(shape)}")
        elif t.shape[-1] != self.nx + 8 or t.numel() != self.m * (self.nx + 8):
            raise ValueError(f"expected a padded slab array [{self.m}, {self.nx + 8}]")
        return t

    def _alpha(self, a):
        torch = self._torch
        na = 2 if self.sys == T7_EULER2D else 1
        if not (isinstance(a, torch.Tensor) and a.is_cuda and a.dtype == torch.float64 and a.numel() >= na):
            raise ValueError(f"alpha values are CUDA float64 tensors of {na} element(s)")
        return a

    def slab_alpha(self, U, alpha_out):
        """max(|u| + c) of the slab's cells (the interior of padded U) into the
        device double tensor alpha_out (one element)."""
        self._check(self.lib.t7_slab_alpha(self.h, _ptr(self._padded(U)), _ptr(self._alpha(alpha_out))),
                    "t7_slab_alpha")
        return alpha_out

    def slab_rhs(self, U, alpha, out=None, want_masks: bool = False):
        """L(U) of the slab's cells (padded U, halos filled) with the global
        alpha (device double tensor: 2D alpha_x, alpha_y); returns dU/dt
        [m, nx] (2D [4, ny, nx]) and, if asked, the masks as euler_rhs's."""
        torch = self._torch
        U = self._padded(U)
        two_d = self.sys == T7_EULER2D
        shape = (4, self.ny, self.nx) if two_d else (self.m, self.nx)
        out = torch.empty(shape, dtype=U.dtype, device=U.device) if out is None else self._dev(out)
        masks = None
        if want_masks:
            nx, ny = self.nx, self.ny
            n = 8 * ny * (nx + 1) + 8 * nx * (ny + 1) if two_d else 2 * self.m * (nx + 1)
            masks = torch.empty(n, dtype=torch.uint8, device=U.device)
        self._check(self.lib.t7_slab_rhs(self.h, _ptr(U), _ptr(self._alpha(alpha)), _ptr(out), _ptr(masks)),
                    "t7_slab_rhs")
        if not want_masks:
            return out
        if two_d:
            k = 8 * self.ny * (self.nx + 1)
            return out, (masks[:k].view(2, 4, self.ny, self.nx + 1), masks[k:].view(2, 4, self.nx, self.ny + 1))
        return out, masks.view(2, self.m, self.nx + 1)

    def slab_stage(self, k: int, Us, U0, out, alpha, dt: float, alpha_out=None):
        """SSP-RK3 stage k of fixed dt on padded slab arrays (see t7_slab_stage)."""
        U0 = None if U0 is None else self._padded(U0)
        alpha_out = None if alpha_out is None else self._alpha(alpha_out)
        self._check(self.lib.t7_slab_stage(self.h, k, _ptr(self._padded(Us)), _ptr(U0), _ptr(self._padded(out)),
                                           _ptr(self._alpha(alpha)), dt, _ptr(alpha_out)), "t7_slab_stage")
        return out

    def rk3_step(self, U, dt: float):
        self._check(self.lib.t7_rk3_step(self.h, _ptr(self._dev(U)), dt), "t7_rk3_step")
        return U

    def run(self, U, cfl: float, t_end: float = math.inf, max_steps: int = 2**31 - 1):
        steps, t = ctypes.c_int(), ctypes.c_double()
        self._check(self.lib.t7_run(self.h, _ptr(self._dev(U)), cfl, t_end, max_steps, ctypes.byref(steps),
                                    ctypes.byref(t)), "t7_run")
        return steps.value, t.value

    def run_host(self, U_host, cfl: float, t_end: float = math.inf, max_steps: int = 2**31 - 1):
        """U_host: a C-contiguous numpy array or a (preferably pinned) CPU torch
        tensor of the context's dtype, [m][nx]; advanced in place."""
        torch = self._torch
        if isinstance(U_host, torch.Tensor):
            if U_host.is_cuda or U_host.dtype != self.dtype or not U_host.is_contiguous():
                raise ValueError(f"expected a contiguous CPU tensor of dtype {self.dtype}")
            ptr = ctypes.c_void_p(U_host.data_ptr())
        else:
            if not (U_host.dtype == self.np_dtype and U_host.flags.c_contiguous):
                raise ValueError(f"expected a C-contiguous {self.np_dtype} array")
            ptr = U_host.ctypes.data_as(ctypes.c_void_p)
        steps, t = ctypes.c_int(), ctypes.c_double()
        self._check(self.lib.t7_run_host(self.h, ptr, cfl, t_end, max_steps, ctypes.byref(steps), ctypes.byref(t)),
                    "t7_run_host")
        return steps.value, t.value

    def rk3_step_static(self, U, dt: float):
        """One RK3 step through t7_rk3_step_static (no allocation, static scratch)."""
        buf = ctypes.create_string_buffer(256)
        st = self.lib.t7_rk3_step_static(ctypes.byref(self.grid), _ptr(self._dev(U)), dt,
                                         ctypes.c_void_p(self.stream.cuda_stream), buf, 256)
        if st != T7_OK:
            raise T7Error(st, f"t7_rk3_step_static: {buf.value.decode()}")
        return U

    # ------------------------------------------------------------ adjoint --
    def euler_rhs_adjoint(self, U, v, out=None):
        """(dL/dU)^T v with the stencil selection and alpha frozen at U."""
        torch = self._torch
        out = torch.empty_like(U) if out is None else self._dev(out)
        self._check(self.lib.t7_euler_rhs_adjoint(self.h, _ptr(self._dev(U)), _ptr(self._dev(v)), _ptr(out)),
                    "t7_euler_rhs_adjoint")
        return out

    def rk3_step_adjoint(self, U, dt: float, lam):
        """Map lam (adjoint of the step result) in place to the adjoint of U."""
        self._check(self.lib.t7_rk3_step_adjoint(self.h, _ptr(self._dev(U)), dt, _ptr(self._dev(lam))),
                    "t7_rk3_step_adjoint")
        return lam

    def tape_bytes(self) -> int:
        b = ctypes.c_size_t()
        self._check(self.lib.t7_tape_bytes(self.h, ctypes.byref(b)), "t7_tape_bytes")
        return b.value

    def rk3_step_record(self, U_in, U_out, dt: float, tape):
        """One fixed-dt step U_in -> U_out recording the stage data into `tape`
        (a CUDA uint8 tensor of tape_bytes(), 256-byte aligned)."""
        self._check(self.lib.t7_rk3_step_record(self.h, _ptr(self._dev(U_in)), _ptr(self._dev(U_out)), dt,
                                                _ptr(tape)), "t7_rk3_step_record")
        return U_out

    def rk3_step_adjoint_recorded(self, U_in, tape, dt: float, lam):
        """Adjoint of a recorded step: lam (adjoint of U_out) -> adjoint of U_in, in place."""
        self._check(self.lib.t7_rk3_step_adjoint_recorded(self.h, _ptr(self._dev(U_in)), _ptr(tape), dt,
                                                          _ptr(self._dev(lam))), "t7_rk3_step_adjoint_recorded")
        return lam

    # ------------------------------------------------------- ragged batch --
    def batch_run(self, U, offsets, dx, t_end: float, cfl: float, max_steps: int = 2**31 - 1,
                  group_warps: int = 0):
        """Advance every tube of the concatenated batch U ([3][sum n]) to t_end in
        one persistent launch.  Returns (steps[ntubes], t[ntubes])."""
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        dxa = np.ascontiguousarray(dx, dtype=np.float64)
        nt = off.size - 1
        steps = np.zeros(nt, np.int32)
        t = np.zeros(nt, np.float64)
        self._check(self.lib.t7_batch_run(self.h, _ptr(self._dev(U)), off.ctypes.data, dxa.ctypes.data, nt, t_end,
                                          cfl, max_steps, group_warps, steps.ctypes.data, t.ctypes.data),
                    "t7_batch_run")
        return steps, t

    def batch_autotune(self, U, offsets, dx, cfl: float, trial_steps: int = 20):
        """Pick group_warps (warps per tube) by timing trial steps; U is not modified.
        Returns (group_warps, trial milliseconds for 1, 2, 4, 8)."""
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        dxa = np.ascontiguousarray(dx, dtype=np.float64)
        g = ctypes.c_int()
        ms = np.zeros(4, np.float32)
        self._check(self.lib.t7_batch_autotune(self.h, _ptr(self._dev(U)), off.ctypes.data, dxa.ctypes.data,
                                               off.size - 1, cfl, trial_steps, ctypes.byref(g), ms.ctypes.data),
                    "t7_batch_autotune")
        return g.value, ms

    def sync(self):
        self._check(self.lib.t7_sync(self.h), "t7_sync")


def probe_fma(kind: int, iters: int = 4096, repeats: int = 3, stream=None) -> tuple[float, float]:
    """Measured FMA rate of the device (t7_probe_fma): (TFLOP/s, ms per launch)."""
    import torch
    lib = load()
    s = stream if stream is not None else torch.cuda.current_stream()
    tf, ms = ctypes.c_double(), ctypes.c_float()
    st = lib.t7_probe_fma(kind, iters, repeats, ctypes.c_void_p(s.cuda_stream), ctypes.byref(tf), ctypes.byref(ms))
    if st != T7_OK:
        raise T7Error(st, "t7_probe_fma failed")
    return tf.value, ms.value


def probe_index_check(i: int, lo: int, hi: int, lib=None) -> tuple[int, bool, bool]:
    """The index check of the checked build on one index (t7_probe_index_check):
    (index an access would use, whether the check latched a failure, whether
    `lib` -- default: the loaded library -- is the checked build)."""
    lib = lib or load()
    idx, flagged, checked = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    st = lib.t7_probe_index_check(i, lo, hi, ctypes.byref(idx), ctypes.byref(flagged), ctypes.byref(checked))
    if st != T7_OK:
        raise T7Error(st, "t7_probe_index_check failed")
    return idx.value, bool(flagged.value), bool(checked.value)
