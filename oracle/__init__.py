"""Plain FP64 CPU oracle for the Strang-split Vlasov step (arXiv:1206.3229, Secs. 2-3).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` are the only users.  The oracle is a small C library (``vlasov_oracle.c``) built with
gcc and loaded through ctypes; it shares no code with the CUDA library and never imports it.

Every function cites the passage of the paper it follows; the C source lists the readings taken
where the paper is silent.  Parity pins for each function live in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vlasov_oracle.c")
_HDR = os.path.join(_HERE, "vlasov_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

HMF, RING, SHEET, FREE = 0, 1, 2, 3
_MODEL_IDS = {"hmf": HMF, "ring": RING, "sheet": SHEET, "free": FREE}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no FP contraction so x86 and Arm agree)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int), ("nx", ctypes.c_long), ("np", ctypes.c_long),
                ("xmin", ctypes.c_double), ("xmax", ctypes.c_double),
                ("pmin", ctypes.c_double), ("pmax", ctypes.c_double),
                ("x_periodic", ctypes.c_int), ("p_periodic", ctypes.c_int),
                ("eps", ctypes.c_double), ("G", ctypes.c_double), ("dt", ctypes.c_double),
                ("spline", ctypes.c_int)]


class _Moments(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("t", "mass", "Mx", "My", "kinetic", "potential", "energy", "l2")]


MOMENT_FIELDS = ("t", "mass", "Mx", "My", "kinetic", "potential", "energy", "l2")

_lib = None
_lock = threading.Lock()


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            pp = ctypes.POINTER(_Params)
            lib.vo_fd2.argtypes = [dp, ctypes.c_long, ctypes.c_int, ctypes.c_double, dp]
            lib.vo_gs2.argtypes = [dp, ctypes.c_long, ctypes.c_int, ctypes.c_double, dp]
            lib.vo_spline_shift.argtypes = [dp, dp, ctypes.c_long, ctypes.c_int, ctypes.c_double,
                                            ctypes.c_double, dp]
            for fn in (lib.vo_advect_x, lib.vo_advect_p):
                fn.argtypes = [pp, dp, dp, dp]
            lib.vo_xshift_cells.argtypes = [pp, dp]
            lib.vo_density.argtypes = [pp, dp, dp]
            lib.vo_force.argtypes = [pp, dp, dp]
            lib.vo_pshift_cells.argtypes = [pp, dp, dp]
            lib.vo_moments_of.argtypes = [pp, dp, ctypes.POINTER(_Moments)]
            lib.vo_entropy.argtypes = [pp, dp]
            lib.vo_entropy.restype = ctypes.c_double
            lib.vo_run.argtypes = [pp, dp, ctypes.c_long, ctypes.POINTER(_Moments)]
            lib.vo_run.restype = ctypes.c_int
            lib.vo_step_parts.argtypes = [pp, dp, dp, dp, dp, dp]
            lib.vo_step_parts.restype = ctypes.c_int
            lib.vo_set_threads.argtypes = [ctypes.c_int]
            lib.vo_set_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass(frozen=True)
class Grid:
    """Problem description shared by the oracle calls (Sec. 3: grid on [xmin,xmax) x [pmin,pmax))."""
    model: str
    nx: int
    np: int
    xmin: float
    xmax: float
    pmin: float
    pmax: float
    x_periodic: bool
    p_periodic: bool
    dt: float
    eps: float = 0.0
    G: float = 1.0
    spline: str = "fd"     # "fd": Eq. (findif); "gs": global spline, Eq. (tridiagsys)

    @property
    def dx(self) -> float:
        return (self.xmax - self.xmin) / self.nx

    @property
    def dp(self) -> float:
        return (self.pmax - self.pmin) / self.np

    def _c(self) -> _Params:
        return _Params(_MODEL_IDS[self.model], self.nx, self.np, self.xmin, self.xmax,
                       self.pmin, self.pmax, int(self.x_periodic), int(self.p_periodic),
                       self.eps, self.G, self.dt, {"fd": 0, "gs": 1}[self.spline])


def set_threads(n: int) -> int:
    """Set the OpenMP thread count of the line sweeps; returns the count in use."""
    return int(_load().vo_set_threads(int(n)))


def fd2(f: np.ndarray, periodic: bool, du: float) -> np.ndarray:
    """Eq. (findif) along a 1-D line: f''_k = (1/du^2) sum_m c_m f_{k+m}."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(f)
    _load().vo_fd2(_ptr(f), f.size, int(periodic), float(du), _ptr(out))
    return out


def gs2(f: np.ndarray, periodic: bool, du: float) -> np.ndarray:
    """Eq. (tridiagsys) along a 1-D line: the global-spline f'' (cyclic system on periodic lines;
    f = f'' = 0 at the neighbour nodes -1 and n of a non-periodic line)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(f)
    _load().vo_gs2(_ptr(f), f.size, int(periodic), float(du), _ptr(out))
    return out


def spline_shift(f: np.ndarray, periodic: bool, du: float, s: float, spline: str = "fd") -> np.ndarray:
    """Eqs. (splinegen, splinecoeffs) on one line: value at the foot i - s of node i, with f'' from
    Eq. (findif) (spline="fd") or Eq. (tridiagsys) (spline="gs")."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    d2 = gs2(f, periodic, du) if spline == "gs" else fd2(f, periodic, du)
    out = np.empty_like(f)
    _load().vo_spline_shift(_ptr(f), _ptr(d2), f.size, int(periodic), float(du), float(s), _ptr(out))
    return out


def advect_x(g: Grid, f: np.ndarray, s_row: np.ndarray) -> np.ndarray:
    """Eq. (step1)/(step4) with per-row displacements s_row (cells)."""
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(g.np, g.nx)
    s_row = np.ascontiguousarray(s_row, dtype=np.float64)
    assert s_row.shape == (g.np,)
    out = np.empty_like(f)
    p = g._c()
    _load().vo_advect_x(ctypes.byref(p), _ptr(f), _ptr(s_row), _ptr(out))
    return out


def advect_p(g: Grid, f: np.ndarray, s_col: np.ndarray) -> np.ndarray:
    """Eq. (step3) with per-column displacements s_col (cells)."""
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(g.np, g.nx)
    s_col = np.ascontiguousarray(s_col, dtype=np.float64)
    assert s_col.shape == (g.nx,)
    out = np.empty_like(f)
    p = g._c()
    _load().vo_advect_p(ctypes.byref(p), _ptr(f), _ptr(s_col), _ptr(out))
    return out


def xshift_cells(g: Grid) -> np.ndarray:
    """Displacement of row j in cells for the half free-streaming step: p_j * (dt/2) / dx."""
    out = np.empty(g.np)
    p = g._c()
    _load().vo_xshift_cells(ctypes.byref(p), _ptr(out))
    return out


def density(g: Grid, f: np.ndarray) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(g.np, g.nx)
    out = np.empty(g.nx)
    p = g._c()
    _load().vo_density(ctypes.byref(p), _ptr(f), _ptr(out))
    return out


def force(g: Grid, rho: np.ndarray) -> np.ndarray:
    """Eq. (meanforce) (Eq. hmfmeanforce for HMF) from the density rho."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    out = np.empty(g.nx)
    p = g._c()
    _load().vo_force(ctypes.byref(p), _ptr(rho), _ptr(out))
    return out


def pshift_cells(g: Grid, F: np.ndarray) -> np.ndarray:
    F = np.ascontiguousarray(F, dtype=np.float64)
    out = np.empty(g.nx)
    p = g._c()
    _load().vo_pshift_cells(ctypes.byref(p), _ptr(F), _ptr(out))
    return out


def moments(g: Grid, f: np.ndarray) -> dict:
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(g.np, g.nx)
    m = _Moments()
    p = g._c()
    _load().vo_moments_of(ctypes.byref(p), _ptr(f), ctypes.byref(m))
    return {k: getattr(m, k) for k in MOMENT_FIELDS}


def entropy(g: Grid, f: np.ndarray) -> float:
    """Eq. (casimirs) with s(f) = -f log f (the entropy of Secs. 4.1-4.2): -dx dp sum_{f > 0} f ln f."""
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(g.np, g.nx)
    p = g._c()
    return float(_load().vo_entropy(ctypes.byref(p), _ptr(f)))


def step_parts(g: Grid, f: np.ndarray) -> dict:
    """One Strang step with its intermediates: f1 (after step 1), F, f2 (after step 3), out."""
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(g.np, g.nx)
    f1, f2, out = np.empty_like(f), np.empty_like(f), np.empty_like(f)
    F = np.empty(g.nx)
    p = g._c()
    rc = _load().vo_step_parts(ctypes.byref(p), _ptr(f), _ptr(f1), _ptr(F), _ptr(f2), _ptr(out))
    if rc != 0:
        raise MemoryError("oracle step failed")
    return {"f1": f1, "F": F, "f2": f2, "out": out}


def run(g: Grid, f0: np.ndarray, nsteps: int, with_moments: bool = True):
    """Sec. 3 steps 1-4 repeated nsteps times.  Returns (f, moments array [nsteps, 8] or None)."""
    f = np.array(f0, dtype=np.float64, copy=True).reshape(g.np, g.nx)
    hist = (_Moments * max(nsteps, 1))() if with_moments else None
    p = g._c()
    rc = _load().vo_run(ctypes.byref(p), _ptr(f), int(nsteps), hist)
    if rc != 0:
        raise MemoryError("oracle run failed")
    if not with_moments:
        return f, None
    arr = np.array([[getattr(hist[n], k) for k in MOMENT_FIELDS] for n in range(nsteps)])
    return f, arr
