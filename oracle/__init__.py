"""FP64 CPU oracle for the TENO7-ext scheme (arXiv:1808.00037).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and bench.py's
CPU-baseline leg may import this package; the product path (the CUDA library
and its binding) never does.  The compute lives in ``teno7_oracle.c`` (plain
C, FP64, no FMA contraction), loaded here through ctypes; this module only
marshals numpy arrays.  It shares no code with the CUDA path.

Parity status of each function (what pins it, see tests/test_oracle_*.py):
  or_coeffs / or_select        -- Table co2 / co3: exact rational re-derivation,
                                  golden copies of the printed tables, and the
                                  "no reconstruction crosses a discontinuity"
                                  rule checked exhaustively over all 32 vectors.
  or_face_bits                 -- hand-computed windows (constant, step), and two
                                  windows whose smallest chi lies just above and
                                  just below C_T, evaluated in exact rationals
                                  (they fail for q = 2, 4, 8, C = 0, a missing
                                  normalisation, a wrong tau or a reversed window).
  teno7_reconstruct / rhs_1d   -- linear 7th-order upwind recovery on smooth
                                  data, measured order >= 6.5, conservation,
                                  mirror symmetry, uniform-flow invariance.
  frame_1d / frame_2d          -- L R = I, A R = R Lambda, Roe's property.
  run_1d                       -- exact Riemann solutions (riemann.py) of the
                                  Sod and Lax tubes; exact shift for advection.
  rhs_2d / run_2d              -- reduces to the 1D scheme on y-independent
                                  data; x/y transpose symmetry.
  alpha_mode(ALPHA_PER_FIELD)  -- per-field alphas: maxima equal to the closed-form
  / alpha_fields_1d                 |u - c|, |u|, |u + c| over the cells, their
  / face_split_1d                   maximum equal to the global alpha bit for bit;
                                  with every field's alpha set to the global one
                                  the RHS equals the global split's to round-off;
                                  conservation; on an entropy wave (u, p
                                  constant) the entropy field's '-' split
                                  vanishes (it does with alpha_1 = |u| only).
  rhs_1d_tl / rk3_step_1d_tl   -- tangent linear with frozen selection and alpha:
  / run_1d_tl                     value parts bit-identical to the primal,
                                  derivative against fourth-order central
                                  differences of the primal (frozen alpha and
                                  masks), Euler's theorem J U = L(U) for the
                                  degree-1 homogeneous frozen scheme.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "teno7_oracle.c"
_LIB_PATH = _HERE / "_build" / "libteno7_oracle.so"

SYS_ADVECTION, SYS_EULER1D, SYS_EULER2D, SYS_BURGERS = 0, 1, 2, 3
BC_PERIODIC, BC_ZERO_GRADIENT = 0, 1
OK, EINVAL, ENONPHYSICAL, ENONFINITE = 0, -1, -3, -4

_lib = None


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (-O2 -ffp-contract=off, no fast-math)."""
    _LIB_PATH.parent.mkdir(exist_ok=True)
    if force or not _LIB_PATH.exists() or _LIB_PATH.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _LIB_PATH.with_suffix(f".{os.getpid()}.tmp.so")
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
             "-o", str(tmp), str(_SRC), "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(str(build()))
        d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        _lib.or_coeffs.argtypes = [p]
        _lib.or_select.argtypes = [i]
        _lib.or_face_bits.argtypes = [p, d, d, p]
        _lib.or_teno7_reconstruct.argtypes = [p, i, i, d, d, p, p, p]
        _lib.or_rhs_1d.argtypes = [i, p, i, d, d, d, d, d, i, i, d, p, p, p]
        _lib.or_rk3_step_1d.argtypes = [i, p, i, d, d, d, d, d, i, i, d]
        _lib.or_cfl_dt_1d.argtypes = [i, p, i, d, d, d, d, p]
        _lib.or_run_1d.argtypes = [i, p, i, d, d, d, d, d, i, i, d, d, d, i, p, p]
        _lib.or_rhs_2d.argtypes = [p, i, i, d, d, d, d, d, d, p, p, p, p, p]
        _lib.or_cfl_dt_2d.argtypes = [p, i, i, d, d, d, d, p]
        _lib.or_rk3_step_2d.argtypes = [p, i, i, d, d, d, d, d, d, p, d]
        _lib.or_run_2d.argtypes = [p, i, i, d, d, d, d, d, d, p, d, d, d, i, p, p]
        _lib.or_frame_1d.argtypes = [p, p, d, p, p]
        _lib.or_alpha_1d.argtypes = [i, p, i, d, d, p]
        _lib.or_alpha_2d.argtypes = [p, i, i, d, p]
        _lib.or_set_scheme.argtypes = [i]
        _lib.or_select5.argtypes = [i]
        _lib.or_coeffs5.argtypes = [p]
        _lib.or_frame_2d.argtypes = [p, p, d, i, p, p]
        _lib.or_rhs_1d_tl.argtypes = [i, p, p, i, d, d, d, i, i, d, p, p, p]
        _lib.or_rk3_step_1d_tl.argtypes = [i, p, p, i, d, d, d, d, d, i, i, d]
        _lib.or_run_1d_tl.argtypes = [i, p, p, i, d, d, d, d, d, i, i, d, i]
        _lib.or_set_alpha_mode.argtypes = [i]
        _lib.or_alpha_fields_1d.argtypes = [i, p, i, d, d, p]
        _lib.or_face_split_1d.argtypes = [i, p, i, d, d, i, i, d, i, p, p]
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleError(RuntimeError):
    pass


def _check(st: int, what: str, strict: bool):
    if st != OK and strict:
        raise OracleError(f"{what}: status {st}")
    return st


SCHEME_TENO7EXT, SCHEME_TENO5 = 0, 1


class scheme:
    """Context manager selecting the oracle's scheme (TENO7-ext by default;
    TENO5 is the baseline the paper compares with)."""

    def __init__(self, which: int):
        self.which = which

    def __enter__(self):
        self.prev = lib().or_get_scheme()
        lib().or_set_scheme(self.which)
        return self

    def __exit__(self, *a):
        lib().or_set_scheme(self.prev)


ALPHA_GLOBAL, ALPHA_PER_FIELD = 0, 1


class alpha_mode:
    """Context manager selecting the oracle's Lax-Friedrichs alpha for the 1D
    systems: one global alpha (default, the paper's choice) or one per
    characteristic field, alpha_k = max_i |lambda_k(U_i)|."""

    def __init__(self, which: int):
        self.which = which

    def __enter__(self):
        self.prev = lib().or_get_alpha_mode()
        lib().or_set_alpha_mode(self.which)
        return self

    def __exit__(self, *a):
        lib().or_set_alpha_mode(self.prev)


def alpha_fields_1d(sys, U, *, gamma=1.4, a=1.0):
    """Per-field alphas max_i |lambda_k(U_i)| (Euler: u - c, u, u + c)."""
    U = _f64(U).reshape(nvars(sys), -1)
    out = np.zeros(nvars(sys))
    _check(lib().or_alpha_fields_1d(sys, _ptr(U), U.shape[1], gamma, a, _ptr(out)), "alpha_fields_1d", True)
    return out


def face_split_1d(sys, U, i, *, gamma=1.4, a=1.0, bc=(BC_PERIODIC, BC_PERIODIC), alpha=-1.0):
    """Characteristic split values of face i+1/2 as the sweep forms them:
    (Pp[m, 7], Pm[m, 7]) -- '+' of field k at cells i-3+t, '-' at i+4-t."""
    U = _f64(U).reshape(nvars(sys), -1)
    m = nvars(sys)
    Pp, Pm = np.zeros((m, 7)), np.zeros((m, 7))
    st = lib().or_face_split_1d(sys, _ptr(U), U.shape[1], gamma, a, bc[0], bc[1], alpha, i, _ptr(Pp), _ptr(Pm))
    _check(st, "face_split_1d", True)
    return Pp, Pm


def coeffs5() -> np.ndarray:
    out = np.zeros(7 * 5)
    lib().or_coeffs5(_ptr(out))
    return out.reshape(7, 5)


def select5(bits: int) -> int:
    return int(lib().or_select5(int(bits)))


# ---------------------------------------------------------------- tables ----
def coeffs() -> np.ndarray:
    out = np.zeros(13 * 7)
    lib().or_coeffs(_ptr(out))
    return out.reshape(13, 7)


def select(delta5: int) -> int:
    return int(lib().or_select(int(delta5)))


def face_bits(w, eps: float, CT: float = 1e-5):
    w = _f64(w)
    beta = np.zeros(3)
    bits = lib().or_face_bits(_ptr(w), eps, CT, _ptr(beta))
    return int(bits), beta


# ------------------------------------------------------ reconstruction ------
def teno7_reconstruct(v_padded, sign: int, eps: float, CT: float = 1e-5, strict: bool = True):
    """v_padded: n+8 values at cells -4..n+3.  Returns (fhat[n+1], d3[n+3], D5[n+1])."""
    v = _f64(v_padded)
    n = v.size - 8
    fhat = np.zeros(n + 1)
    d3 = np.zeros(n + 3, np.uint8)
    D5 = np.zeros(n + 1, np.uint8)
    st = lib().or_teno7_reconstruct(_ptr(v), n, int(sign), eps, CT, _ptr(fhat), _ptr(d3), _ptr(D5))
    _check(st, "teno7_reconstruct", strict)
    return fhat, d3, D5


# ------------------------------------------------------------------ 1D ------
def nvars(sys: int) -> int:
    return {SYS_ADVECTION: 1, SYS_BURGERS: 1, SYS_EULER1D: 3, SYS_EULER2D: 4}[sys]


def rhs_1d(sys, U, dx, *, gamma=1.4, a=1.0, CT=1e-5, eps=-1.0, bc=(BC_PERIODIC, BC_PERIODIC),
           alpha=-1.0, want_masks=False, strict=True):
    """L(U) for U of shape [m, n].  Returns (dUdt, alpha, masks[2, m, n+1] or None)."""
    U = _f64(U)
    m = nvars(sys)
    U = U.reshape(m, -1)
    n = U.shape[1]
    out = np.zeros_like(U)
    masks = np.zeros((2, m, n + 1), np.uint8) if want_masks else None
    al = np.zeros(1)
    st = lib().or_rhs_1d(sys, _ptr(U), n, dx, gamma, a, CT, eps, bc[0], bc[1], alpha, _ptr(out),
                         _ptr(masks), _ptr(al))
    _check(st, "rhs_1d", strict)
    return out, float(al[0]), masks


def rk3_step_1d(sys, U, dx, dt, *, gamma=1.4, a=1.0, CT=1e-5, eps=-1.0, bc=(BC_PERIODIC, BC_PERIODIC),
                strict=True):
    U = _f64(U).copy()
    m = nvars(sys)
    U = U.reshape(m, -1)
    st = lib().or_rk3_step_1d(sys, _ptr(U), U.shape[1], dx, gamma, a, CT, eps, bc[0], bc[1], dt)
    _check(st, "rk3_step_1d", strict)
    return U


def cfl_dt_1d(sys, U, dx, cfl, *, gamma=1.4, a=1.0):
    U = _f64(U)
    m = nvars(sys)
    U = U.reshape(m, -1)
    dt = np.zeros(1)
    st = lib().or_cfl_dt_1d(sys, _ptr(U), U.shape[1], dx, gamma, a, cfl, _ptr(dt))
    _check(st, "cfl_dt_1d", True)
    return float(dt[0])


# ------------------------------------------------------ tangent linear ----
def rhs_1d_tl(sys, U, dU, dx, alpha, masks, *, gamma=1.4, a=1.0, bc=(BC_PERIODIC, BC_PERIODIC)):
    """(L(U), (dL/dU) dU) with alpha and the selection `masks` ([2, m, n+1]
    Delta codes, as rhs_1d returns them for U) frozen.  TENO7-ext only."""
    U = _f64(U)
    m = nvars(sys)
    U = U.reshape(m, -1)
    dU = _f64(dU).reshape(m, -1)
    n = U.shape[1]
    masks = np.ascontiguousarray(masks, dtype=np.uint8)
    if masks.shape != (2, m, n + 1):
        raise ValueError("masks must be [2, m, n + 1]")
    L, dL = np.zeros_like(U), np.zeros_like(U)
    st = lib().or_rhs_1d_tl(sys, _ptr(U), _ptr(dU), n, dx, gamma, a, bc[0], bc[1], alpha, _ptr(masks), _ptr(L),
                            _ptr(dL))
    _check(st, "rhs_1d_tl", True)
    return L, dL


def rk3_step_1d_tl(sys, U, dU, dx, dt, *, gamma=1.4, a=1.0, CT=1e-5, eps=-1.0, bc=(BC_PERIODIC, BC_PERIODIC)):
    """One SSP-RK3 step of fixed dt and its tangent along dU (each stage's
    alpha and selection frozen at the primal stage state).  Returns (U', dU')."""
    m = nvars(sys)
    U = _f64(U).copy().reshape(m, -1)
    dU = _f64(dU).copy().reshape(m, -1)
    st = lib().or_rk3_step_1d_tl(sys, _ptr(U), _ptr(dU), U.shape[1], dx, gamma, a, CT, eps, bc[0], bc[1], dt)
    _check(st, "rk3_step_1d_tl", True)
    return U, dU


def run_1d_tl(sys, U, dU, dx, dt, nsteps, *, gamma=1.4, a=1.0, CT=1e-5, eps=-1.0, bc=(BC_PERIODIC, BC_PERIODIC)):
    """nsteps tangent-linear RK3 steps of fixed dt.  Returns (U_final, dU_final)."""
    m = nvars(sys)
    U = _f64(U).copy().reshape(m, -1)
    dU = _f64(dU).copy().reshape(m, -1)
    st = lib().or_run_1d_tl(sys, _ptr(U), _ptr(dU), U.shape[1], dx, gamma, a, CT, eps, bc[0], bc[1], dt,
                            int(nsteps))
    _check(st, "run_1d_tl", True)
    return U, dU


def alpha_1d(sys, U, *, gamma=1.4, a=1.0):
    """max_i of the largest characteristic speed over the cells of U[m, n]."""
    U = _f64(U)
    U = U.reshape(nvars(sys), -1)
    out = np.zeros(1)
    st = lib().or_alpha_1d(sys, _ptr(U), U.shape[1], gamma, a, _ptr(out))
    _check(st, "alpha_1d", True)
    return float(out[0])


def run_1d(sys, U, dx, *, t_end, cfl=0.5, dt_fixed=-1.0, max_steps=1 << 30, gamma=1.4, a=1.0, CT=1e-5,
           eps=-1.0, bc=(BC_PERIODIC, BC_PERIODIC), strict=True):
    """Returns (U_final[m, n], steps, t, status)."""
    U = _f64(U).copy()
    m = nvars(sys)
    U = U.reshape(m, -1)
    steps = np.zeros(1, np.int32)
    t = np.zeros(1)
    st = lib().or_run_1d(sys, _ptr(U), U.shape[1], dx, gamma, a, CT, eps, bc[0], bc[1], cfl, dt_fixed,
                         t_end, int(min(max_steps, 2**31 - 1)), _ptr(steps), _ptr(t))
    _check(st, "run_1d", strict)
    return U, int(steps[0]), float(t[0]), st


# ------------------------------------------------------------------ 2D ------
def rhs_2d(U, dx, dy, *, gamma=1.4, CT=1e-5, eps=(-1.0, -1.0),
           bc=(BC_ZERO_GRADIENT,) * 4, alpha=None, want_masks=False, strict=True):
    """U: [4, ny, nx].  Returns (dUdt, (alpha_x, alpha_y), masks or None).
    masks = (xm[2, 4, ny, nx+1], ym[2, 4, nx, ny+1])."""
    U = _f64(U)
    _, ny, nx = U.shape
    out = np.zeros_like(U)
    bcv = np.asarray(bc, np.int32)
    al = np.zeros(2)
    ain = None if alpha is None else _f64(alpha)
    buf = np.zeros(8 * ny * (nx + 1) + 8 * nx * (ny + 1), np.uint8) if want_masks else None
    st = lib().or_rhs_2d(_ptr(U), nx, ny, dx, dy, gamma, CT, eps[0], eps[1], _ptr(bcv), _ptr(ain),
                         _ptr(out), _ptr(buf), _ptr(al))
    _check(st, "rhs_2d", strict)
    masks = None
    if want_masks:
        k = 8 * ny * (nx + 1)
        masks = (buf[:k].reshape(2, 4, ny, nx + 1), buf[k:].reshape(2, 4, nx, ny + 1))
    return out, (float(al[0]), float(al[1])), masks


def alpha_2d(U, *, gamma=1.4):
    """(max |u|+c, max |v|+c) over the cells of U[4, ny, nx]."""
    U = _f64(U)
    _, ny, nx = U.shape
    out = np.zeros(2)
    st = lib().or_alpha_2d(_ptr(U), nx, ny, gamma, _ptr(out))
    _check(st, "alpha_2d", True)
    return float(out[0]), float(out[1])


def cfl_dt_2d(U, dx, dy, cfl, *, gamma=1.4):
    U = _f64(U)
    _, ny, nx = U.shape
    dt = np.zeros(1)
    st = lib().or_cfl_dt_2d(_ptr(U), nx, ny, dx, dy, gamma, cfl, _ptr(dt))
    _check(st, "cfl_dt_2d", True)
    return float(dt[0])


def run_2d(U, dx, dy, *, t_end=np.inf, cfl=0.4, dt_fixed=-1.0, max_steps=1 << 30, gamma=1.4, CT=1e-5,
           eps=(-1.0, -1.0), bc=(BC_ZERO_GRADIENT,) * 4, strict=True):
    U = _f64(U).copy()
    _, ny, nx = U.shape
    bcv = np.asarray(bc, np.int32)
    steps = np.zeros(1, np.int32)
    t = np.zeros(1)
    st = lib().or_run_2d(_ptr(U), nx, ny, dx, dy, gamma, CT, eps[0], eps[1], _ptr(bcv), cfl, dt_fixed,
                         t_end, int(min(max_steps, 2**31 - 1)), _ptr(steps), _ptr(t))
    _check(st, "run_2d", strict)
    return U, int(steps[0]), float(t[0]), st


# ---------------------------------------------------------------- frames ----
def frame_1d(UL, UR, gamma=1.4):
    L = np.zeros(9)
    R = np.zeros(9)
    st = lib().or_frame_1d(_ptr(_f64(UL)), _ptr(_f64(UR)), gamma, _ptr(L), _ptr(R))
    return L.reshape(3, 3), R.reshape(3, 3), st


def frame_2d(UL, UR, direction, gamma=1.4):
    L = np.zeros(16)
    R = np.zeros(16)
    st = lib().or_frame_2d(_ptr(_f64(UL)), _ptr(_f64(UR)), gamma, int(direction), _ptr(L), _ptr(R))
    return L.reshape(4, 4), R.reshape(4, 4), st
