"""ctypes binding of libvlasov.so (include/vlasov.h): argument marshalling only.

Every step of the solver runs in the library's CUDA kernels.  The binding fails loudly when the
library is missing or no CUDA device is present; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build
from .inputs import Workload

HMF, RING, SHEET, FREE = 0, 1, 2, 3
F64, F32, F64_NATIVE, FX64, BF16 = 0, 1, 2, 3, 4
MODELS = {"hmf": HMF, "ring": RING, "sheet": SHEET, "free": FREE}
PRECISIONS = {"f64": F64, "f32": F32, "f64_native": F64_NATIVE, "fx64": FX64, "bf16": BF16}

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ESTATE, ERANGE = 0, -1, -2, -3, -4, -5, -6

EXPORTED = ("vlasov_create", "vlasov_set_f", "vlasov_set_f_device", "vlasov_get_f", "vlasov_get_f_device",
            "vlasov_step", "vlasov_moments", "vlasov_substep", "vlasov_density_force", "vlasov_sync",
            "vlasov_destroy", "vlasov_last_error", "vlasov_kernels_per_step", "vlasov_step_timed",
            "vlasov_xshift_density_noalloc", "vlasov_batch_create", "vlasov_batch_footprint",
            "vlasov_batch_admit", "vlasov_batch_step", "vlasov_batch_slot_steps", "vlasov_batch_get",
            "vlasov_batch_release", "vlasov_batch_destroy", "vlasov_serve", "vlasov_launches",
            "vlasov_set_fused_x", "vlasov_fused_x", "vlasov_batch_create_shaped", "vlasov_batch_shape_of",
            "vlasov_batch_autotune", "vlasov_casimirs", "vlasov_set_spline", "vlasov_spline",
            "vlasov_init_waterbag", "vlasov_test_expire_wait", "vlasov_set_ring_method", "vlasov_ring_method",
            "vlasov_ring_timings")

RING_METHODS = {"direct": 1, "fixed": 2, "fft": 3, "fft_f32": 4, "tensor": 5}
N_RING_METHODS = 6

SPLINES = {"fd": 0, "gs": 1}   # Eq. (findif) (the paper's method) / global spline, Eq. (tridiagsys)


class VlasovError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"vlasov error {code}: {msg}")
        self.code = code


class Domain(ctypes.Structure):
    _fields_ = [("xmin", ctypes.c_double), ("xmax", ctypes.c_double),
                ("pmin", ctypes.c_double), ("pmax", ctypes.c_double),
                ("x_periodic", ctypes.c_int), ("p_periodic", ctypes.c_int),
                ("eps", ctypes.c_double), ("G", ctypes.c_double),
                ("precision", ctypes.c_int), ("stream", ctypes.c_void_p)]


class Moments(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("mass", ctypes.c_double), ("Mx", ctypes.c_double),
                ("My", ctypes.c_double), ("kinetic", ctypes.c_double), ("potential", ctypes.c_double),
                ("energy", ctypes.c_double), ("step", ctypes.c_longlong)]


MOMENT_FIELDS = ("t", "mass", "Mx", "My", "kinetic", "potential", "energy")


class Request(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int), ("Nx", ctypes.c_int), ("Np", ctypes.c_int),
                ("xmin", ctypes.c_double), ("xmax", ctypes.c_double), ("pmin", ctypes.c_double),
                ("pmax", ctypes.c_double), ("x_periodic", ctypes.c_int), ("eps", ctypes.c_double),
                ("G", ctypes.c_double), ("dt", ctypes.c_double), ("init", ctypes.c_int), ("x0", ctypes.c_double),
                ("p0", ctypes.c_double), ("noise", ctypes.c_double), ("amp", ctypes.c_double),
                ("seed", ctypes.c_ulonglong), ("steps", ctypes.c_int), ("arrival_s", ctypes.c_double)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("steps", ctypes.c_int), ("arrival_s", ctypes.c_double),
                ("admit_s", ctypes.c_double), ("done_s", ctypes.c_double), ("last", Moments), ("first", Moments)]


class ServeOptions(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int), ("max_n", ctypes.c_int), ("mem_budget_bytes", ctypes.c_longlong),
                ("max_inflight", ctypes.c_int), ("precision", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("autotune", ctypes.c_int)]


class BatchShape(ctypes.Structure):
    """vlasov_batch_shape: x-shift rows per CTA, p-shift tiles per CTA of the largest grid."""
    _fields_ = [("rows_per_cta", ctypes.c_int), ("tiles_per_cta", ctypes.c_int)]

    def as_tuple(self) -> tuple[int, int]:
        return (self.rows_per_cta, self.tiles_per_cta)


# candidate order of vlasov_batch_autotune
AUTOTUNE_CANDIDATES = [(r, t) for r in (8, 16, 32, 64) for t in (2, 4, 8, 16)]


def request_from_workload(w: Workload, steps: int | None = None, arrival_s: float = 0.0) -> Request:
    """Batched-form request for a workload description (p always zero outside)."""
    return Request(MODELS[w.model], w.nx, w.np, w.xmin, w.xmax, w.pmin, w.pmax, int(w.x_periodic), w.eps, w.G,
                   w.dt, 0 if w.init == "box" else 1, w.x0, w.p0, w.noise, w.mode_amp, w.seed,
                   int(w.steps if steps is None else steps), float(arrival_s))


def moments_row(m: Moments) -> list[float]:
    return [getattr(m, f) for f in MOMENT_FIELDS] + [m.step]


def _batch_precision(precision) -> int:
    p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    if p not in (F32, FX64):
        raise ValueError("batched form: precision 'f32' or 'fx64'")
    return p


class Batch:
    """vlasov_batch_*: many simulations advanced by one launch per sub-step (FP32 or FX64 storage)."""

    def __init__(self, slots: int, max_n: int, mem_budget_bytes: int, stream: int | None = None,
                 precision: str | int = "f32", shape: tuple[int, int] | None = None):
        lib = load()
        h = ctypes.c_void_p()
        sh = BatchShape(*shape) if shape is not None else None
        _check(lib.vlasov_batch_create_shaped(int(slots), int(max_n), int(mem_budget_bytes),
                                              _batch_precision(precision), ctypes.c_void_p(stream) if stream else None,
                                              ctypes.byref(sh) if sh is not None else None, ctypes.byref(h)))
        self._h, self._lib = h, lib

    @property
    def shape(self) -> tuple[int, int]:
        sh = BatchShape()
        _check(self._lib.vlasov_batch_shape_of(self._h, ctypes.byref(sh)))
        return sh.as_tuple()

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.vlasov_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def admit(self, req: Request, f0: np.ndarray | None = None) -> int:
        slot = ctypes.c_int(-1)
        if f0 is not None:
            f0 = np.ascontiguousarray(f0, dtype=np.float64)
            assert f0.size == req.Nx * req.Np
        _check(self._lib.vlasov_batch_admit(self._h, ctypes.byref(req), _dptr(f0) if f0 is not None else None,
                                            ctypes.byref(slot)))
        return slot.value

    def step(self, n: int = 1):
        _check(self._lib.vlasov_batch_step(self._h, int(n)))

    def steps_done(self, slot: int) -> int:
        v = ctypes.c_int(0)
        _check(self._lib.vlasov_batch_slot_steps(self._h, int(slot), ctypes.byref(v)))
        return v.value

    def get(self, slot: int, nx: int, np_: int, max_records: int = 4096):
        f = np.empty((np_, nx), dtype=np.float64)
        buf = (Moments * max(max_records, 1))()
        cnt = ctypes.c_int(0)
        _check(self._lib.vlasov_batch_get(self._h, int(slot), _dptr(f), buf, int(max_records), ctypes.byref(cnt)))
        m = np.array([moments_row(buf[k]) for k in range(cnt.value)], dtype=np.float64).reshape(-1, 8)
        return f, m

    def release(self, slot: int):
        _check(self._lib.vlasov_batch_release(self._h, int(slot)))


def batch_footprint(req: Request, precision: str | int = "f32") -> int:
    return int(load().vlasov_batch_footprint(ctypes.byref(req), _batch_precision(precision)))


def batch_autotune(max_n: int, precision: str | int = "f32", stream: int | None = None):
    """vlasov_batch_autotune: the fastest launch shape for batches up to max_n on this GPU (kept for
    the process) and every candidate's ms per batched step, keyed by AUTOTUNE_CANDIDATES."""
    lib = load()
    best = BatchShape()
    ms = (ctypes.c_double * len(AUTOTUNE_CANDIDATES))()
    _check(lib.vlasov_batch_autotune(int(max_n), _batch_precision(precision), ctypes.c_void_p(stream) if stream else None,
                                     ctypes.byref(best), ms))
    return best.as_tuple(), dict(zip(AUTOTUNE_CANDIDATES, [float(v) for v in ms]))


def serve(reqs: list[Request], slots: int, mem_budget_bytes: int, max_n: int = 0, max_inflight: int = 4,
          stream: int | None = None, precision: str | int = "f32", autotune: bool = False):
    """vlasov_serve: continuous batching of a request stream ("f32" or "fx64" slots).  Returns
    (results, makespan_s)."""
    lib = load()
    arr = (Request * len(reqs))(*reqs)
    res = (Result * max(len(reqs), 1))()
    prec = _batch_precision(precision)
    opt = ServeOptions(int(slots), int(max_n), int(mem_budget_bytes), int(max_inflight), prec,
                       ctypes.c_void_p(stream) if stream else None, 1 if autotune else 0)
    mk = ctypes.c_double(0.0)
    _check(lib.vlasov_serve(arr, len(reqs), ctypes.byref(opt), res, ctypes.byref(mk)))
    return [res[k] for k in range(len(reqs))], mk.value

_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libvlasov.so (building it first if it is missing or stale and nvcc is available)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libvlasov.so not found at {path}; run paper_1206_3229_gb300/build.py")
        lib = ctypes.CDLL(path)
        vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
        lib.vlasov_create.argtypes = [ip, ip, ip, ctypes.POINTER(Domain), ctypes.c_double, ctypes.POINTER(vp)]
        lib.vlasov_set_f.argtypes = [vp, dp]
        lib.vlasov_set_f_device.argtypes = [vp, vp]
        lib.vlasov_test_expire_wait.argtypes = [vp, ctypes.c_longlong]
        lib.vlasov_set_ring_method.argtypes = [vp, ip]
        lib.vlasov_ring_method.argtypes = [vp]
        lib.vlasov_ring_timings.argtypes = [vp, ip, dp]
        lib.vlasov_init_waterbag.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_ulonglong, ip, ctypes.c_double]
        lib.vlasov_get_f.argtypes = [vp, dp]
        lib.vlasov_get_f_device.argtypes = [vp, vp]
        lib.vlasov_step.argtypes = [vp, ip]
        lib.vlasov_moments.argtypes = [vp, ctypes.POINTER(Moments), ip, ctypes.POINTER(ctypes.c_int)]
        lib.vlasov_substep.argtypes = [vp, ip, dp]
        lib.vlasov_density_force.argtypes = [vp, dp, dp]
        lib.vlasov_sync.argtypes = [vp]
        lib.vlasov_destroy.argtypes = [vp]
        lib.vlasov_destroy.restype = None
        lib.vlasov_last_error.argtypes = []
        lib.vlasov_last_error.restype = ctypes.c_char_p
        lib.vlasov_kernels_per_step.argtypes = [vp]
        lib.vlasov_launches.argtypes = [vp, ip]
        lib.vlasov_set_fused_x.argtypes = [vp, ip]
        lib.vlasov_fused_x.argtypes = [vp]
        lib.vlasov_set_spline.argtypes = [vp, ip]
        lib.vlasov_spline.argtypes = [vp]
        lib.vlasov_step_timed.argtypes = [vp, ip, dp, ip, ctypes.POINTER(ctypes.c_int)]
        lib.vlasov_xshift_density_noalloc.argtypes = [vp, vp, vp, ip, ip, ctypes.c_double, ctypes.c_double, ip,
                                                      vp, vp]
        lib.vlasov_batch_create.argtypes = [ip, ip, ctypes.c_longlong, ip, vp, ctypes.POINTER(vp)]
        lib.vlasov_batch_footprint.argtypes = [ctypes.POINTER(Request), ip]
        lib.vlasov_batch_create_shaped.argtypes = [ip, ip, ctypes.c_longlong, ip, vp, ctypes.POINTER(BatchShape),
                                                   ctypes.POINTER(vp)]
        lib.vlasov_batch_shape_of.argtypes = [vp, ctypes.POINTER(BatchShape)]
        lib.vlasov_batch_autotune.argtypes = [ip, ip, vp, ctypes.POINTER(BatchShape), dp]
        lib.vlasov_casimirs.argtypes = [vp, dp, dp]
        lib.vlasov_batch_admit.argtypes = [vp, ctypes.POINTER(Request), dp, ctypes.POINTER(ctypes.c_int)]
        lib.vlasov_batch_step.argtypes = [vp, ip]
        lib.vlasov_batch_slot_steps.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_int)]
        lib.vlasov_batch_get.argtypes = [vp, ip, dp, ctypes.POINTER(Moments), ip, ctypes.POINTER(ctypes.c_int)]
        lib.vlasov_batch_release.argtypes = [vp, ip]
        lib.vlasov_batch_destroy.argtypes = [vp]
        lib.vlasov_batch_destroy.restype = None
        lib.vlasov_serve.argtypes = [ctypes.POINTER(Request), ip, ctypes.POINTER(ServeOptions),
                                     ctypes.POINTER(Result), ctypes.POINTER(ctypes.c_double)]
        for name in EXPORTED:
            if name not in ("vlasov_destroy", "vlasov_last_error", "vlasov_batch_destroy"):
                getattr(lib, name).restype = ctypes.c_int
        lib.vlasov_batch_footprint.restype = ctypes.c_longlong
        lib.vlasov_launches.restype = ctypes.c_longlong
        _lib = lib
        return lib


def _check(rc: int):
    if rc != OK:
        raise VlasovError(rc, _lib.vlasov_last_error().decode(errors="replace"))


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def xshift_density_noalloc(dev_fin: int, dev_fout: int, dev_rho: int, nx: int, np_: int, pmin: float,
                           pmax: float, x_periodic: bool, dev_disp: int, stream: int | None = None):
    """vlasov_xshift_density_noalloc: one x-shift with density for callers that cannot allocate
    device memory (all pointers are caller-owned device buffers; the library's fixed scratch is used)."""
    lib = load()
    _check(lib.vlasov_xshift_density_noalloc(ctypes.c_void_p(dev_fin), ctypes.c_void_p(dev_fout),
                                             ctypes.c_void_p(dev_rho), int(nx), int(np_), float(pmin), float(pmax),
                                             int(bool(x_periodic)), ctypes.c_void_p(dev_disp),
                                             ctypes.c_void_p(stream) if stream else None))


class Sim:
    """One simulation handle (vlasov_create ... vlasov_destroy)."""

    def __init__(self, model: str | int, nx: int, np_: int, xmin: float, xmax: float, pmin: float,
                 pmax: float, dt: float, x_periodic: bool = True, p_periodic: bool = False,
                 eps: float = 0.0, G: float = 1.0, precision: str | int = "f64", stream: int | None = None):
        lib = load()
        self.model = MODELS[model] if isinstance(model, str) else int(model)
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.nx, self.np = int(nx), int(np_)
        dom = Domain(xmin, xmax, pmin, pmax, int(x_periodic), int(p_periodic), eps, G, self.precision,
                     ctypes.c_void_p(stream) if stream else None)
        h = ctypes.c_void_p()
        _check(lib.vlasov_create(self.model, self.nx, self.np, ctypes.byref(dom), float(dt), ctypes.byref(h)))
        self._h = h
        self._lib = lib

    @classmethod
    def from_workload(cls, w: Workload, precision: str = "f64", stream: int | None = None) -> "Sim":
        return cls(w.model, w.nx, w.np, w.xmin, w.xmax, w.pmin, w.pmax, w.dt, w.x_periodic, w.p_periodic,
                   w.eps, w.G, precision, stream)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.vlasov_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self) -> int:
        return self._h.value

    def set_f(self, f: np.ndarray):
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.size == self.nx * self.np
        _check(self._lib.vlasov_set_f(self._h, _dptr(f)))

    def set_f_device(self, dev_ptr: int):
        _check(self._lib.vlasov_set_f_device(self._h, ctypes.c_void_p(dev_ptr)))

    def init_waterbag(self, x0: float, p0: float, noise: float = 0.0, seed: int = 0, mode: int = 0,
                      mode_amp: float = 0.0):
        """vlasov_init_waterbag: a Sec. 4 waterbag written on the device (mode 0 box with seeded
        noise, mode 1 homogeneous with a cos mode), normalised to unit mass."""
        _check(self._lib.vlasov_init_waterbag(self._h, float(x0), float(p0), float(noise), int(seed) & (2**64 - 1),
                                              int(mode), float(mode_amp)))

    def init_workload(self, w: Workload):
        """The initial state of a workload description, generated on the device."""
        if w.init == "box":
            self.init_waterbag(w.x0, w.p0, w.noise, w.seed, 0, 0.0)
        elif w.init == "mode":
            self.init_waterbag(w.x0, w.p0, 0.0, 0, 1, w.mode_amp)
        else:
            raise ValueError(f"unknown init {w.init!r}")

    def get_f(self, out: np.ndarray | None = None) -> np.ndarray:
        if out is None:
            out = np.empty((self.np, self.nx), dtype=np.float64)
        _check(self._lib.vlasov_get_f(self._h, _dptr(out)))
        return out

    def get_f_device(self, dev_ptr: int):
        _check(self._lib.vlasov_get_f_device(self._h, ctypes.c_void_p(dev_ptr)))

    def step(self, n: int = 1):
        _check(self._lib.vlasov_step(self._h, int(n)))

    def moments(self, max_records: int = 4096) -> np.ndarray:
        """Records since the previous call, as an array [n, 8]: t, mass, Mx, My, kinetic, potential, energy, step."""
        buf = (Moments * max(max_records, 1))()
        cnt = ctypes.c_int(0)
        _check(self._lib.vlasov_moments(self._h, buf, int(max_records), ctypes.byref(cnt)))
        return np.array([[getattr(buf[k], f) for f in MOMENT_FIELDS] + [buf[k].step] for k in range(cnt.value)],
                        dtype=np.float64).reshape(-1, 8)

    def substep(self, axis: int, disp: np.ndarray):
        disp = np.ascontiguousarray(disp, dtype=np.float64)
        assert disp.size == (self.np if axis == 0 else self.nx)
        _check(self._lib.vlasov_substep(self._h, int(axis), _dptr(disp)))

    def density_force(self):
        rho = np.empty(self.nx)
        F = np.empty(self.nx)
        _check(self._lib.vlasov_density_force(self._h, _dptr(rho), _dptr(F)))
        return rho, F

    def sync(self):
        _check(self._lib.vlasov_sync(self._h))

    @property
    def ring_method(self) -> str:
        m = int(self._lib.vlasov_ring_method(self._h))
        return {v: k for k, v in RING_METHODS.items()}.get(m, "")

    @ring_method.setter
    def ring_method(self, name: str):
        _check(self._lib.vlasov_set_ring_method(self._h, RING_METHODS[name]))

    def ring_timings(self, reps: int = 50) -> dict:
        """vlasov_ring_timings: microseconds per force launch of each ring method that can run."""
        us = np.zeros(N_RING_METHODS)
        _check(self._lib.vlasov_ring_timings(self._h, int(reps), _dptr(us)))
        return {k: float(us[v]) for k, v in RING_METHODS.items() if us[v] > 0}

    def test_expire_wait(self, limit_ns: int):
        """vlasov_test_expire_wait: enqueue a bounded device wait that must expire (failure-path check)."""
        _check(self._lib.vlasov_test_expire_wait(self._h, int(limit_ns)))

    def casimirs(self) -> tuple[float, float]:
        """(entropy, integral of f^2) of the current f (vlasov_casimirs)."""
        e, q = ctypes.c_double(0.0), ctypes.c_double(0.0)
        _check(self._lib.vlasov_casimirs(self._h, ctypes.byref(e), ctypes.byref(q)))
        return e.value, q.value

    def kernels_per_step(self) -> int:
        return int(self._lib.vlasov_kernels_per_step(self._h))

    def launches(self, n: int) -> int:
        """Kernel launches that step(n) enqueues."""
        return int(self._lib.vlasov_launches(self._h, int(n)))

    @property
    def fused_x(self) -> bool:
        """Whether step(n >= 2) fuses the second x half-shift of a step with the first of the next."""
        return bool(self._lib.vlasov_fused_x(self._h))

    @fused_x.setter
    def fused_x(self, on: bool):
        _check(self._lib.vlasov_set_fused_x(self._h, 1 if on else 0))

    @property
    def spline(self) -> str:
        """"fd" (f'' by Eq. findif, the default) or "gs" (the global spline of Eq. tridiagsys)."""
        return "gs" if self._lib.vlasov_spline(self._h) == SPLINES["gs"] else "fd"

    @spline.setter
    def spline(self, name: str):
        _check(self._lib.vlasov_set_spline(self._h, SPLINES[name]))

    def step_timed(self, n: int) -> np.ndarray:
        """Mean milliseconds of each launch slot of a step over n eager steps (see vlasov.h)."""
        out = np.zeros(16)
        cnt = ctypes.c_int(0)
        _check(self._lib.vlasov_step_timed(self._h, int(n), _dptr(out), 16, ctypes.byref(cnt)))
        return out[:cnt.value].copy()

    def slot_names(self) -> list[str]:
        """Names of the step_timed slots (for n >= 2 when fused_x)."""
        hmf_cta = self.model == HMF and self.precision in (FX64, BF16, F32) and self.nx * self.np <= 1 << 24 \
            and self.spline == "fd"
        if self.fused_x and self.model == RING and self.ring_method == "fixed":
            # the end state's moments and the next force: reductions and convolutions merged, the
            # force launch also writing the p-shift filters
            return ["xshift_fused", "reduce_moments_density", "ring_potential_force_filters", "pshift_step3"]
        # HMF with FP32-class storage: the p-shift forms its filters itself (no filter launch)
        filt = [] if (hmf_cta and self.precision in (BF16, F32)) else ["force_filters"]
        if self.fused_x:
            names = ["xshift_fused", "reduce_moments"]
            if self.model == RING:
                names.append("ring_potential")
            if hmf_cta:
                return names + filt + ["pshift_step3"]
            names.append("reduce_density")
            if self.model == RING:
                names.append("ring_force")
            return names + ["pshift_filters", "pshift_step3"]
        if hmf_cta:
            return ["xshift_step1"] + filt + ["pshift_step3", "xshift_step4", "reduce_moments"]
        names = ["xshift_step1", "reduce_density"]
        if self.model == RING and self.ring_method == "fixed":
            names.append("ring_force_filters")
        else:
            if self.model == RING:
                names.append("ring_force")
            names.append("pshift_filters")
        names += ["pshift_step3", "xshift_step4", "reduce_moments"]
        if self.model == RING:
            names.append("ring_potential")
        return names
