"""FP64 CPU oracle of the HYDRO directionally split Godunov scheme (§1, Fig. 5).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, the package smoke
check (``__graft_entry__.smoke``) and the CPU-baseline leg of ``bench.py`` may
import this module.  It loads ``liboracle.so`` built from ``hydro_oracle.c``
(plain C, gcc, no FMA contraction) and shares nothing with the CUDA path.

Every function here is a thin ctypes marshaller; all arithmetic is in the C
file, whose comments state the definition each step follows.

Pins: every entry point is pinned by ``tests/test_oracle_*.py`` (exact Sod
star state, closed forms of the Riemann problem, jump conditions and fan
invariants, uniform-state preservation, conservation, transpose symmetry,
stencil footprint, reduction to the scalar MUSCL-Hancock scheme, convergence
to the exact Sod profile).  The Sedov-blast workload itself has no closed
form pinned here: for it, the scheme is pinned only through the properties
above.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hydro_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None

BC_REFLECT, BC_TRANSMISSIVE, BC_PERIODIC = 0, 1, 2


RIEMANN_EXACT, RIEMANN_TWO_SHOCK = 0, 1
SLOPE_MINMOD, SLOPE_MC, SLOPE_NONE = 0, 1, 2
TRACE_MUSCL_HANCOCK, TRACE_CHARACTERISTIC = 0, 1


class Params(ctypes.Structure):
    _fields_ = [
        ("gamma", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("niter", ctypes.c_int),
        ("rho_floor", ctypes.c_double),
        ("c_floor", ctypes.c_double),
        ("riemann", ctypes.c_int),
        ("slope", ctypes.c_int),
        ("trace", ctypes.c_int),
    ]


def params(gamma=1.4, cfl=0.8, niter=10, rho_floor=1e-10, c_floor=1e-10,
           riemann=RIEMANN_EXACT, slope=SLOPE_MINMOD, trace=TRACE_MUSCL_HANCOCK) -> Params:
    """Scheme parameters; riemann (exact / two-shock pressure function),
    slope (minmod / monotonized central / none) and trace (MUSCL-Hancock /
    characteristic tracing) select the variants."""
    return Params(gamma, cfl, niter, rho_floor, c_floor, riemann, slope, trace)


def build(force: bool = False, omp: bool = False) -> str:
    """Compile liboracle.so next to the source (gcc, -ffp-contract=off); with
    omp=True the same source with -fopenmp into liboracle_omp.so (lines of a
    sweep shared among threads, bit-identical results)."""
    out = _LIB_OMP if omp else _LIB
    with _lock:
        if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
            tmp = out + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                   "-fPIC", "-shared", *(["-fopenmp"] if omp else []), "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, out)
    return out


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_P = ctypes.POINTER(Params)


def _bind(L):
    L.orc_riemann_star.argtypes = [_P, _D, _D, _D, _D]
    L.orc_sample.argtypes = [_P, _D, _D, ctypes.c_double, ctypes.c_double, ctypes.c_double, _D]
    L.orc_interface_flux.argtypes = [_P, _D, _D, _D]
    L.orc_run.argtypes = [_P, ctypes.c_int, ctypes.c_int, ctypes.c_double, _I, _D,
                          ctypes.c_long, ctypes.c_int, _D, _D]
    L.orc_run.restype = ctypes.c_int
    L.orc_sweep.argtypes = [_P, ctypes.c_int, ctypes.c_int, ctypes.c_double, _I, _D,
                            ctypes.c_int, ctypes.c_double]
    L.orc_sweep.restype = ctypes.c_int
    L.orc_cfl_dt.argtypes = [_P, ctypes.c_int, ctypes.c_int, ctypes.c_double, _D]
    L.orc_cfl_dt.restype = ctypes.c_double
    L.orc_conservation.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _D, _D]
    L.orc_godunov_line.argtypes = [_P, ctypes.c_int, ctypes.c_double, _D, _D]
    L.orc_godunov_line.restype = ctypes.c_int
    L.orc_trace.argtypes = [_P, ctypes.c_double, _D, _D, _D, _D, _D]
    L.orc_cons_to_prim.argtypes = [_P, _D, _D]
    L.orc_set_threads.argtypes = [ctypes.c_int]
    L.orc_set_threads.restype = ctypes.c_int
    return L


def lib():
    """The loaded oracle library.  ORACLE_LIB names another build of the same
    source (used only by the mutation test, which plants mistakes in copies)."""
    global _lib
    if _lib is None:
        path = os.environ.get("ORACLE_LIB")
        if not path:
            path = build()
        _lib = _bind(ctypes.CDLL(path))
    return _lib


def lib_omp():
    """The -fopenmp build of the same source (lines of a sweep shared among
    threads; bit-identical to lib())."""
    global _lib_omp
    if _lib_omp is None:
        _lib_omp = _bind(ctypes.CDLL(build(omp=True)))
    return _lib_omp


def set_threads(n: int) -> int:
    """Threads of the OpenMP build's sweeps (0: its default); returns the
    number it will use."""
    return int(lib_omp().orc_set_threads(int(n)))


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _vec4(w) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(w, dtype=np.float64).reshape(4))
    return a


def riemann_star(wl, wr, P: Params | None = None):
    """(p*, u*) for primitive states (rho, u_n, u_t, p)."""
    P = P or params()
    a, b = _vec4(wl), _vec4(wr)
    ps, us = ctypes.c_double(), ctypes.c_double()
    lib().orc_riemann_star(ctypes.byref(P), _dp(a), _dp(b), ctypes.byref(ps), ctypes.byref(us))
    return ps.value, us.value


def sample(wl, wr, pstar, ustar, xi, P: Params | None = None) -> np.ndarray:
    """Primitive state of the Riemann solution at x/t = xi."""
    P = P or params()
    a, b = _vec4(wl), _vec4(wr)
    w = np.zeros(4)
    lib().orc_sample(ctypes.byref(P), _dp(a), _dp(b), pstar, ustar, xi, _dp(w))
    return w


def interface_flux(wl, wr, P: Params | None = None) -> np.ndarray:
    P = P or params()
    a, b = _vec4(wl), _vec4(wr)
    f = np.zeros(4)
    lib().orc_interface_flux(ctypes.byref(P), _dp(a), _dp(b), _dp(f))
    return f


def trace(dtdx, wm, w0, wp, P: Params | None = None):
    P = P or params()
    a, b, c = _vec4(wm), _vec4(w0), _vec4(wp)
    wl, wr = np.zeros(4), np.zeros(4)
    lib().orc_trace(ctypes.byref(P), dtdx, _dp(a), _dp(b), _dp(c), _dp(wl), _dp(wr))
    return wl, wr


def cons_to_prim(u, P: Params | None = None) -> np.ndarray:
    P = P or params()
    a = _vec4(u)
    w = np.zeros(4)
    lib().orc_cons_to_prim(ctypes.byref(P), _dp(a), _dp(w))
    return w


def godunov_line(line: np.ndarray, dtdx: float, P: Params | None = None) -> np.ndarray:
    """line: (n+4, 4) conserved (rho, m_n, m_t, E), cells -2..n+1 -> (n, 4)."""
    P = P or params()
    a = np.ascontiguousarray(line, dtype=np.float64)
    n = a.shape[0] - 4
    out = np.zeros((n, 4))
    rc = lib().orc_godunov_line(ctypes.byref(P), n, dtdx, _dp(a), _dp(out))
    if rc:
        raise RuntimeError(f"orc_godunov_line failed: {rc}")
    return out


def _bc(bc) -> ctypes.Array:
    return (ctypes.c_int * 4)(*[int(b) for b in bc])


def run(U: np.ndarray, h: float, bc, nsteps: int, step0: int = 0, dt_override=None,
        P: Params | None = None, check: bool = True, threads: int | None = None):
    """Advance a copy of U ([4, ny, nx] FP64) by nsteps; returns (U_new, dts, rc).
    threads: None runs the single-threaded build; n >= 0 the OpenMP build
    with n threads (0: its default), which gives the same bits."""
    P = P or params()
    L = lib()
    if threads is not None:
        L = lib_omp()
        L.orc_set_threads(int(threads))
    a = np.array(U, dtype=np.float64, order="C", copy=True)
    _, ny, nx = a.shape
    dts = np.zeros(max(nsteps, 1))
    ov = None
    if dt_override is not None:
        ov = np.ascontiguousarray(dt_override, dtype=np.float64)
        if ov.shape[0] < nsteps:
            raise ValueError("dt_override shorter than nsteps")
    rc = L.orc_run(ctypes.byref(P), nx, ny, h, _bc(bc), _dp(a), step0, nsteps,
                       _dp(ov) if ov is not None else None, _dp(dts))
    if check and rc not in (0,):
        raise RuntimeError(f"orc_run failed: {rc}")
    return a, dts[:nsteps], rc


def sweep(U: np.ndarray, h: float, bc, direction: int, dt: float,
          P: Params | None = None) -> np.ndarray:
    P = P or params()
    a = np.array(U, dtype=np.float64, order="C", copy=True)
    _, ny, nx = a.shape
    rc = lib().orc_sweep(ctypes.byref(P), nx, ny, h, _bc(bc), _dp(a), direction, dt)
    if rc:
        raise RuntimeError(f"orc_sweep failed: {rc}")
    return a


def cfl_dt(U: np.ndarray, h: float, P: Params | None = None) -> float:
    P = P or params()
    a = np.ascontiguousarray(U, dtype=np.float64)
    _, ny, nx = a.shape
    return lib().orc_cfl_dt(ctypes.byref(P), nx, ny, h, _dp(a))


def conservation(U: np.ndarray, h: float) -> np.ndarray:
    a = np.ascontiguousarray(U, dtype=np.float64)
    _, ny, nx = a.shape
    s = np.zeros(4)
    lib().orc_conservation(nx, ny, h, _dp(a), _dp(s))
    return s
