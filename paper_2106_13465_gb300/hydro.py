"""Python binding of the libhydro C ABI (include/hydro.h): ctypes marshalling
only.  Every step of the scheme runs in the library's CUDA kernels; this
module never computes any part of it.  If libhydro.so is missing or cannot be
loaded, every call raises: there is no fallback path.

Functions keep the C names (hydro_init, hydro_set_state, hydro_step,
hydro_get_state, hydro_cfl_dt, ...).  `Context` is a small convenience
wrapper that owns one hydro_ctx and raises HydroError on a non-OK status.
Arrays are numpy FP64 [4, ny, nx] on the host, or any object exposing a CUDA
device pointer through `data_ptr()` (e.g. a CUDA torch tensor) on the device.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

HYDRO_OK, HYDRO_EINVAL, HYDRO_ENOMEM, HYDRO_ECUDA, HYDRO_ENEGATIVE, HYDRO_ETIMEOUT = range(6)
BC_REFLECT, BC_TRANSMISSIVE, BC_PERIODIC = 0, 1, 2
PREC_FP32, PREC_FP64 = 32, 64
RIEMANN_EXACT, RIEMANN_TWO_SHOCK = 0, 1
SLOPE_MINMOD, SLOPE_MC, SLOPE_NONE = 0, 1, 2
TRACE_MUSCL_HANCOCK, TRACE_CHARACTERISTIC = 0, 1
STATUS_NAMES = {0: "HYDRO_OK", 1: "HYDRO_EINVAL", 2: "HYDRO_ENOMEM", 3: "HYDRO_ECUDA",
                4: "HYDRO_ENEGATIVE", 5: "HYDRO_ETIMEOUT"}

# every symbol the header declares (checked by the CPU test of the ABI)
EXPORTS = ("hydro_init", "hydro_destroy", "hydro_set_tuning", "hydro_set_wait_limit", "hydro_set_state",
           "hydro_get_state", "hydro_set_rows", "hydro_get_rows", "hydro_step", "hydro_step_dt", "hydro_step_profiled", "hydro_cfl_dt", "hydro_get_time",
           "hydro_get_step", "hydro_set_step", "hydro_set_time",
           "hydro_conservation", "hydro_conservation_noalloc", "hydro_get_stats",
           "hydro_last_error", "hydro_version")


class hydro_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("h", ctypes.c_double),
                ("bc", ctypes.c_int * 4)]


class hydro_params(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("gamma", ctypes.c_double), ("cfl", ctypes.c_double),
                ("niter_riemann", ctypes.c_int), ("rho_floor", ctypes.c_double),
                ("c_floor", ctypes.c_double), ("ngrids", ctypes.c_int),
                ("grids", ctypes.POINTER(hydro_grid)), ("cuda_stream", ctypes.c_void_p),
                ("riemann_solver", ctypes.c_int), ("slope_type", ctypes.c_int),
                ("trace_type", ctypes.c_int)]


class hydro_tuning(ctypes.Structure):
    _fields_ = [("tile_len", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("graph_steps", ctypes.c_int), ("span_len", ctypes.c_int), ("fused", ctypes.c_int)]


class hydro_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_longlong), ("riemann_fp64", ctypes.c_longlong),
                ("status_flags", ctypes.c_uint), ("kernel_launches", ctypes.c_longlong),
                ("wait_site", ctypes.c_int), ("wait_tile", ctypes.c_int)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libhydro.so (building it first if asked and absent)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"libhydro.so not built at {path}")
        _build.build()
    L = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp, D = ctypes.c_void_p, P(ctypes.c_double)
    L.hydro_init.argtypes = [P(hydro_params), P(vp)]
    L.hydro_destroy.argtypes = [vp]
    L.hydro_destroy.restype = None
    L.hydro_set_tuning.argtypes = [vp, P(hydro_tuning)]
    L.hydro_set_wait_limit.argtypes = [vp, ctypes.c_longlong]
    L.hydro_set_state.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int]
    L.hydro_get_state.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int]
    L.hydro_set_rows.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int]
    L.hydro_get_rows.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int]
    L.hydro_step.argtypes = [vp, ctypes.c_int, D]
    L.hydro_step_dt.argtypes = [vp, ctypes.c_int, D, D]
    L.hydro_step_profiled.argtypes = [vp, ctypes.c_int, D]
    L.hydro_cfl_dt.argtypes = [vp, ctypes.c_int, D]
    L.hydro_get_time.argtypes = [vp, ctypes.c_int, D]
    L.hydro_get_step.argtypes = [vp, P(ctypes.c_longlong)]
    L.hydro_set_step.argtypes = [vp, ctypes.c_longlong]
    L.hydro_set_time.argtypes = [vp, ctypes.c_int, ctypes.c_double]
    L.hydro_conservation.argtypes = [vp, ctypes.c_int, D]
    L.hydro_conservation_noalloc.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, vp, vp]
    L.hydro_conservation_noalloc.restype = ctypes.c_int
    L.hydro_get_stats.argtypes = [vp, P(hydro_stats)]
    L.hydro_last_error.argtypes = [vp]
    L.hydro_last_error.restype = ctypes.c_char_p
    L.hydro_version.argtypes = []
    L.hydro_version.restype = ctypes.c_char_p
    for name in ("hydro_init", "hydro_set_tuning", "hydro_set_wait_limit", "hydro_set_state", "hydro_get_state",
                 "hydro_set_rows", "hydro_get_rows",
                 "hydro_step", "hydro_step_dt", "hydro_step_profiled", "hydro_cfl_dt",
                 "hydro_get_time", "hydro_get_step", "hydro_set_step", "hydro_set_time",
                 "hydro_conservation", "hydro_get_stats"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


class HydroError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ---- the C functions under their own names ---------------------------------
def hydro_init(params: hydro_params):
    ctx = ctypes.c_void_p()
    st = load().hydro_init(ctypes.byref(params), ctypes.byref(ctx))
    return st, ctx


def hydro_destroy(ctx) -> None:
    load().hydro_destroy(ctx)


def hydro_set_tuning(ctx, tuning: hydro_tuning) -> int:
    return load().hydro_set_tuning(ctx, ctypes.byref(tuning))


def hydro_set_wait_limit(ctx, polls: int) -> int:
    return load().hydro_set_wait_limit(ctx, polls)


def hydro_set_state(ctx, grid: int, U_ptr: int, on_device: int) -> int:
    return load().hydro_set_state(ctx, grid, ctypes.c_void_p(U_ptr), on_device)


def hydro_get_state(ctx, grid: int, U_ptr: int, on_device: int) -> int:
    return load().hydro_get_state(ctx, grid, ctypes.c_void_p(U_ptr), on_device)


def hydro_set_rows(ctx, grid: int, row0: int, nrows: int, U_ptr: int, on_device: int) -> int:
    return load().hydro_set_rows(ctx, grid, row0, nrows, ctypes.c_void_p(U_ptr), on_device)


def hydro_get_rows(ctx, grid: int, row0: int, nrows: int, U_ptr: int, on_device: int) -> int:
    return load().hydro_get_rows(ctx, grid, row0, nrows, ctypes.c_void_p(U_ptr), on_device)


def hydro_step(ctx, nsteps: int, dt_override: np.ndarray | None = None) -> int:
    return load().hydro_step(ctx, nsteps, None if dt_override is None else _dptr(dt_override))


def hydro_step_dt(ctx, nsteps: int, dt_override, dt_used) -> int:
    return load().hydro_step_dt(ctx, nsteps, None if dt_override is None else _dptr(dt_override),
                                None if dt_used is None else _dptr(dt_used))


def hydro_step_profiled(ctx, nsteps: int, kernel_ms: np.ndarray) -> int:
    return load().hydro_step_profiled(ctx, nsteps, _dptr(kernel_ms))


def hydro_cfl_dt(ctx, grid: int):
    v = ctypes.c_double()
    return load().hydro_cfl_dt(ctx, grid, ctypes.byref(v)), v.value


def hydro_get_time(ctx, grid: int):
    v = ctypes.c_double()
    return load().hydro_get_time(ctx, grid, ctypes.byref(v)), v.value


def hydro_get_step(ctx):
    v = ctypes.c_longlong()
    return load().hydro_get_step(ctx, ctypes.byref(v)), v.value


def hydro_set_step(ctx, step: int) -> int:
    return load().hydro_set_step(ctx, step)


def hydro_set_time(ctx, grid: int, t: float) -> int:
    return load().hydro_set_time(ctx, grid, t)


def hydro_conservation(ctx, grid: int):
    s = np.zeros(4)
    return load().hydro_conservation(ctx, grid, _dptr(s)), s


def hydro_conservation_noalloc(U_ptr: int, nx: int, ny: int, h: float, sums_ptr: int,
                               stream: int | None = None) -> int:
    """Totals of a device state [4, ny, nx] into a device array of 4 doubles,
    without allocating (see include/hydro.h)."""
    return load().hydro_conservation_noalloc(ctypes.c_void_p(U_ptr), nx, ny, h,
                                             ctypes.c_void_p(sums_ptr), ctypes.c_void_p(stream or 0))


def hydro_get_stats(ctx):
    s = hydro_stats()
    return load().hydro_get_stats(ctx, ctypes.byref(s)), s


def hydro_last_error(ctx=None) -> str:
    r = load().hydro_last_error(ctx)
    return r.decode() if r else ""


def hydro_version() -> str:
    return load().hydro_version().decode()


# ---- convenience wrapper -----------------------------------------------------
def make_params(grids, precision: int = PREC_FP64, gamma: float = 1.4, cfl: float = 0.8,
                niter: int = 10, rho_floor: float = 1e-10, c_floor: float = 1e-10,
                stream: int | None = None, riemann: int = RIEMANN_EXACT, slope: int = SLOPE_MINMOD,
                trace: int = TRACE_MUSCL_HANCOCK):
    """grids: iterable of (nx, ny, h, (bc_xlo, bc_xhi, bc_ylo, bc_yhi));
    riemann / slope / trace select the scheme variants (include/hydro.h)."""
    grids = list(grids)
    arr = (hydro_grid * len(grids))()
    for k, (nx, ny, h, bc) in enumerate(grids):
        arr[k].nx, arr[k].ny, arr[k].h = int(nx), int(ny), float(h)
        for q in range(4):
            arr[k].bc[q] = int(bc[q])
    p = hydro_params(precision, gamma, cfl, niter, rho_floor, c_floor, len(grids),
                     ctypes.cast(arr, ctypes.POINTER(hydro_grid)), stream or None, riemann, slope, trace)
    return p, arr


class Context:
    """One hydro_ctx: `Context([(nx, ny, h, bc), ...], precision=64)`."""

    def __init__(self, grids, precision: int = PREC_FP64, stream: int | None = None, **kw):
        self.grids = [(int(g[0]), int(g[1]), float(g[2]), tuple(g[3])) for g in grids]
        self._params, self._arr = make_params(self.grids, precision, stream=stream, **kw)
        st, ctx = hydro_init(self._params)
        if st != HYDRO_OK:
            raise HydroError(st, hydro_last_error(None))
        self.ctx = ctx
        self.precision = precision

    def _check(self, st: int) -> None:
        if st != HYDRO_OK:
            raise HydroError(st, hydro_last_error(self.ctx))

    def close(self) -> None:
        if getattr(self, "ctx", None):
            hydro_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_tuning(self, tile_len: int = 0, ctas_per_sm: int = 0, graph_steps: int = 20,
                   span_len: int = 0, fused: int = 0) -> None:
        self._check(hydro_set_tuning(self.ctx, hydro_tuning(tile_len, ctas_per_sm, graph_steps, span_len,
                                                            fused)))

    def set_wait_limit(self, polls: int = -1) -> None:
        """Polls of a TMA completion before a sweep gives up (-1: default)."""
        self._check(hydro_set_wait_limit(self.ctx, polls))

    def set_state(self, grid: int, U) -> None:
        if hasattr(U, "data_ptr"):
            self._check(hydro_set_state(self.ctx, grid, U.data_ptr(), 1))
        else:
            nx, ny = self.grids[grid][:2]
            a = np.ascontiguousarray(U, dtype=np.float64)
            if a.shape != (4, ny, nx):
                raise ValueError(f"state of grid {grid} must be [4, {ny}, {nx}]")
            self._check(hydro_set_state(self.ctx, grid, a.ctypes.data, 0))

    def get_state(self, grid: int, out=None):
        nx, ny = self.grids[grid][:2]
        if out is not None and hasattr(out, "data_ptr"):
            self._check(hydro_get_state(self.ctx, grid, out.data_ptr(), 1))
            return out
        a = np.empty((4, ny, nx)) if out is None else out
        self._check(hydro_get_state(self.ctx, grid, a.ctypes.data, 0))
        return a

    def set_rows(self, grid: int, row0: int, U) -> None:
        """Write rows [row0, row0 + U.shape[1]) of a grid (U: [4, nrows, nx])."""
        if hasattr(U, "data_ptr"):
            self._check(hydro_set_rows(self.ctx, grid, row0, int(U.shape[1]), U.data_ptr(), 1))
        else:
            a = np.ascontiguousarray(U, dtype=np.float64)
            if a.ndim != 3 or a.shape[0] != 4 or a.shape[2] != self.grids[grid][0]:
                raise ValueError("rows must be [4, nrows, nx]")
            self._check(hydro_set_rows(self.ctx, grid, row0, a.shape[1], a.ctypes.data, 0))

    def get_rows(self, grid: int, row0: int, nrows: int, out=None):
        """Read rows [row0, row0 + nrows) of a grid as [4, nrows, nx]."""
        nx = self.grids[grid][0]
        if out is not None and hasattr(out, "data_ptr"):
            self._check(hydro_get_rows(self.ctx, grid, row0, nrows, out.data_ptr(), 1))
            return out
        a = np.empty((4, nrows, nx)) if out is None else out
        self._check(hydro_get_rows(self.ctx, grid, row0, nrows, a.ctypes.data, 0))
        return a

    def step(self, nsteps: int, dt_override=None, record_dt: bool = False):
        ov = None
        if dt_override is not None:
            ov = np.ascontiguousarray(dt_override, dtype=np.float64).reshape(-1)
            if ov.size < nsteps * len(self.grids):
                raise ValueError("dt_override needs nsteps * ngrids values")
        if record_dt:
            used = np.zeros(nsteps * len(self.grids))
            self._check(hydro_step_dt(self.ctx, nsteps, ov, used))
            return used.reshape(nsteps, len(self.grids))
        self._check(hydro_step(self.ctx, nsteps, ov))
        return None

    def step_profiled(self, nsteps: int) -> np.ndarray:
        """Run nsteps (no graph) and return [nsteps, 3] launch durations in ms
        (dt prologue, first sweep, second sweep)."""
        ms = np.zeros(3 * nsteps)
        self._check(hydro_step_profiled(self.ctx, nsteps, ms))
        return ms.reshape(nsteps, 3)

    def cfl_dt(self, grid: int = 0) -> float:
        st, v = hydro_cfl_dt(self.ctx, grid)
        self._check(st)
        return v

    def time(self, grid: int = 0) -> float:
        st, v = hydro_get_time(self.ctx, grid)
        self._check(st)
        return v

    def get_step(self) -> int:
        st, v = hydro_get_step(self.ctx)
        self._check(st)
        return v

    def set_step(self, step: int) -> None:
        self._check(hydro_set_step(self.ctx, step))

    def set_time(self, grid: int, t: float) -> None:
        self._check(hydro_set_time(self.ctx, grid, t))

    def conservation(self, grid: int = 0) -> np.ndarray:
        st, s = hydro_conservation(self.ctx, grid)
        self._check(st)
        return s

    def stats(self) -> dict:
        st, s = hydro_get_stats(self.ctx)
        self._check(st)
        return {"steps": s.steps, "riemann_fp64": s.riemann_fp64, "status_flags": s.status_flags,
                "kernel_launches": s.kernel_launches, "wait_site": s.wait_site, "wait_tile": s.wait_tile}
