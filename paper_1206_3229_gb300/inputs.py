"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and by the oracle.

This module holds no arithmetic of the method: only the problem descriptions (grid, domain, time
step, model constants) of the workloads and the initial distributions (waterbags of Sec. 4 of
arXiv:1206.3229, with optional seeded noise or a cos-theta mode), generated with numpy.

Noise: xi_ij = 2*u - 1 with u the top 53 bits of the (j*nx + i + 1)-th output of SplitMix64
(Steele, Lea & Flood, OOPSLA 2014) seeded with ``seed`` -- a counter-based draw, so any cell's
value is known without generating the others.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counter: np.ndarray) -> np.ndarray:
    """The counter-th output (counter >= 1) of SplitMix64 started at state ``seed``."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + np.asarray(counter, dtype=np.uint64) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, counter: np.ndarray) -> np.ndarray:
    """u in [0, 1): top 53 bits of the SplitMix64 output divided by 2^53."""
    return (splitmix64(seed, counter) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclass(frozen=True)
class Workload:
    """One simulation: model, grid, domain, step and initial state recipe."""
    name: str
    model: str            # "hmf" | "ring" | "sheet" | "free"
    nx: int
    np: int
    xmin: float
    xmax: float
    pmin: float
    pmax: float
    x_periodic: bool
    p_periodic: bool
    dt: float
    steps: int
    eps: float = 0.0
    G: float = 1.0
    init: str = "box"     # "box": |x|<x0 and |p|<p0 ; "mode": homogeneous in x with a cos mode
    x0: float = 1.0
    p0: float = 1.0
    noise: float = 0.0
    seed: int = 0
    mode_amp: float = 0.0

    @property
    def dx(self) -> float:
        return (self.xmax - self.xmin) / self.nx

    @property
    def dp(self) -> float:
        return (self.pmax - self.pmin) / self.np

    @property
    def cells(self) -> int:
        return self.nx * self.np

    def resized(self, nx: int, np_: int | None = None, **kw) -> "Workload":
        return replace(self, nx=nx, np=np_ if np_ is not None else nx, **kw)


PI = math.pi

# The four single-grid workloads (x fastest; theta periodic for HMF/ring; p zero outside).
HMF_256 = Workload("hmf_256_fp64", "hmf", 256, 256, -PI, PI, -4.0, 4.0, True, False, 0.1, 200,
                   init="box", x0=1.895, p0=1.0, noise=1e-4, seed=1)
HMF_4096_UNSTABLE = Workload("hmf_4096_unstable", "hmf", 4096, 4096, -PI, PI, -2.0, 2.0, True, False,
                             0.05, 1000, init="mode", x0=PI, p0=math.sqrt(6.0 * (0.55 - 0.5)),
                             mode_amp=1e-6)
RING_2048 = Workload("ring_2048", "ring", 2048, 2048, -PI, PI, -3.0, 3.0, True, False, 0.05, 1000,
                     eps=0.01, init="box", x0=1.0, p0=0.8, noise=1e-4, seed=3)
SHEET_4096 = Workload("sheet_4096", "sheet", 4096, 4096, -8.0, 8.0, -4.0, 4.0, False, False, 0.02, 2000,
                      G=1.0, init="box", x0=1.0, p0=0.5, noise=1e-4, seed=4)

WORKLOADS = {w.name: w for w in (HMF_256, HMF_4096_UNSTABLE, RING_2048, SHEET_4096)}


def nodes(w: Workload):
    """Grid nodes x_i = xmin + i dx and p_j = pmin + j dp (endpoint excluded)."""
    x = w.xmin + np.arange(w.nx, dtype=np.float64) * w.dx
    p = w.pmin + np.arange(w.np, dtype=np.float64) * w.dp
    return x, p


def initial_state(w: Workload) -> np.ndarray:
    """Initial f[j, i] (shape np x nx, float64), renormalised to unit mass dx*dp*sum f = 1.

    box : f = 1/(4 x0 p0) where |x_i| < x0 and |p_j| < p0, times (1 + noise*xi_ij).  x0 >= half
          the x-extent means every column (a homogeneous waterbag).
    mode: f = [|p_j| < p0] / (2 p0 L) * (1 + mode_amp cos x_i), L = x-extent.
    """
    x, p = nodes(w)
    X, P = np.meshgrid(x, p)  # shapes (np, nx)
    half_x = 0.5 * (w.xmax - w.xmin)
    if w.init == "box":
        inx = np.ones_like(X, dtype=bool) if w.x0 >= half_x else (np.abs(X) < w.x0)
        f = np.where(inx & (np.abs(P) < w.p0), 1.0 / (4.0 * w.x0 * w.p0), 0.0)
        if w.noise:
            idx = np.arange(w.cells, dtype=np.uint64).reshape(w.np, w.nx) + np.uint64(1)
            xi = 2.0 * uniform01(w.seed, idx) - 1.0
            f = f * (1.0 + w.noise * xi)
    elif w.init == "mode":
        L = w.xmax - w.xmin
        f = np.where(np.abs(P) < w.p0, 1.0 / (2.0 * w.p0 * L), 0.0) * (1.0 + w.mode_amp * np.cos(X))
    else:
        raise ValueError(f"unknown init {w.init!r}")
    mass = w.dx * w.dp * f.sum()
    return np.ascontiguousarray(f / mass)


# Domains and time steps per model for the serving stream (those of the single-grid workloads).
SERVING_DOMAINS = {
    "hmf": dict(xmin=-PI, xmax=PI, pmin=-2.0, pmax=2.0, x_periodic=True, dt=0.05, eps=0.0, G=1.0),
    "ring": dict(xmin=-PI, xmax=PI, pmin=-3.0, pmax=3.0, x_periodic=True, dt=0.05, eps=0.01, G=1.0),
    "sheet": dict(xmin=-8.0, xmax=8.0, pmin=-4.0, pmax=4.0, x_periodic=False, dt=0.02, eps=0.0, G=1.0),
}


def serving_stream(n: int = 512, seed: int = 5, sizes=(256, 512, 1024, 2048), steps=(100, 2000),
                   rate_per_s: float = 50.0, step_scale: float = 1.0):
    """A seeded Poisson stream of simulation requests: model uniform over HMF/ring/sheet, square grid
    uniform over `sizes`, waterbag half-widths x0 ~ U[0.5, pi], p0 ~ U[0.3, 1.5], noise 1e-4, steps
    ~ U[steps] (times step_scale), exponential inter-arrival times of mean 1/rate_per_s.
    Returns a list of (Workload, steps, arrival_s)."""
    rng = np.random.default_rng(seed)
    out = []
    t = 0.0
    models = ("hmf", "ring", "sheet")
    for q in range(n):
        m = models[int(rng.integers(0, 3))]
        N = int(sizes[int(rng.integers(0, len(sizes)))])
        x0 = float(rng.uniform(0.5, PI))
        p0 = float(rng.uniform(0.3, 1.5))
        st = max(1, int(round(int(rng.integers(steps[0], steps[1] + 1)) * step_scale)))
        t += float(rng.exponential(1.0 / rate_per_s))
        d = SERVING_DOMAINS[m]
        w = Workload(f"req{q}_{m}_{N}", m, N, N, d["xmin"], d["xmax"], d["pmin"], d["pmax"], d["x_periodic"], False,
                     d["dt"], st, eps=d["eps"], G=d["G"], init="box", x0=x0, p0=p0, noise=1e-4,
                     seed=seed * 100000 + q)
        out.append((w, st, t))
    return out
