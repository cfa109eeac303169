"""The global-spline variant (Sec. 3, Eq. tridiagsys: the comparison method of Tables 1-2) on the GPU,
through the C ABI, against the oracle's tridiagonal solve, element by element.

Bars as for the spline of Eq. findif in the same arithmetic: one IEEE FP64 sweep to rounding
(1e-13 max|f|), 200 HMF steps at 256^2 to 1e-12 max f, FP32 storage to 5e-6 max|f| per sweep
(64-tap filter in FP32) and |dM| <= 1e-5 over the run.
"""
import numpy as np
import pytest

import oracle as O
from paper_1206_3229_gb300 import inputs as I
from paper_1206_3229_gb300 import vlasov as V

pytestmark = pytest.mark.gpu

TOL = {"f64_native": 1e-13, "f32": 5e-6}


def grid_gs(w: I.Workload) -> O.Grid:
    return O.Grid(w.model, w.nx, w.np, w.xmin, w.xmax, w.pmin, w.pmax, w.x_periodic, w.p_periodic,
                  w.dt, w.eps, w.G, spline="gs")


def make_gs(w, prec):
    s = V.Sim.from_workload(w, precision=prec)
    s.spline = "gs"
    return s


CASES = [
    ("periodic_x_ragged", 200, 328, True, False),
    ("zero_x_ragged", 200, 328, False, False),
    ("periodic_p", 96, 144, True, True),
    ("smallest", 64, 64, False, False),
]


@pytest.mark.parametrize("prec", ["f64_native", "f32"])
@pytest.mark.parametrize("name,nx,np_,xper,pper", CASES)
def test_gs_x_sweep_matches_oracle(prec, name, nx, np_, xper, pper):
    w = I.Workload(name, "free", nx, np_, -1.0, 1.0, -2.0, 2.0, xper, pper, 0.1, 1)
    rng = np.random.default_rng(nx + np_)
    f = rng.uniform(0.0, 1.0, (np_, nx))
    for disp in (rng.uniform(-30, 30, np_), np.linspace(-3.3, 2.7, np_), np.round(rng.uniform(-9, 9, np_)),
                 np.full(np_, nx + 5.5)):
        with make_gs(w, prec) as s:
            s.set_f(f)
            s.substep(0, disp)
            got = s.get_f()
        want = O.advect_x(grid_gs(w), f, disp)
        assert np.max(np.abs(got - want)) <= TOL[prec] * max(np.abs(want).max(), 1.0), name


@pytest.mark.parametrize("prec", ["f64_native", "f32"])
@pytest.mark.parametrize("name,nx,np_,xper,pper", CASES)
def test_gs_p_sweep_matches_oracle(prec, name, nx, np_, xper, pper):
    w = I.Workload(name, "free", nx, np_, -1.0, 1.0, -2.0, 2.0, xper, pper, 0.1, 1)
    rng = np.random.default_rng(3 * nx + np_)
    f = rng.uniform(0.0, 1.0, (np_, nx))
    x = np.arange(nx)
    cases = [
        4.0 * np.sin(2 * np.pi * x / nx) + 0.3,          # smooth, like a mean-field force (staged rows)
        rng.uniform(-40, 40, nx),                          # spread inside a tile (staged rows)
        rng.uniform(-150, 150, nx),                        # spread past the staging rows (global reads)
        np.full(nx, -1.0 * np_ - 7.5),                     # everything moved out of the grid
    ]
    for disp in cases:
        with make_gs(w, prec) as s:
            s.set_f(f)
            s.substep(1, disp)
            got = s.get_f()
        want = O.advect_p(grid_gs(w), f, disp)
        assert np.max(np.abs(got - want)) <= TOL[prec] * max(np.abs(want).max(), 1.0), name


def test_gs_hmf_256_fp64_200_steps_matches_oracle():
    w = I.HMF_256
    f0 = I.initial_state(w)
    fo, mo = O.run(grid_gs(w), f0, w.steps)
    with make_gs(w, "f64_native") as s:
        s.set_f(f0)
        s.step(w.steps)
        mg = s.moments()
        fg = s.get_f()
    assert np.max(np.abs(fg - fo)) <= 1e-12 * fo.max()
    for col in (1, 2, 3, 4, 5, 6):
        assert np.max(np.abs(mg[:, col] - mo[:, col])) <= 1e-12, col


@pytest.mark.parametrize("w,steps", [
    (I.RING_2048.resized(128, 128), 40),
    (I.SHEET_4096.resized(128, 256), 40),
], ids=["ring", "sheet"])
def test_gs_models_fp64_steps_match_oracle(w, steps):
    f0 = I.initial_state(w)
    fo, mo = O.run(grid_gs(w), f0, steps)
    with make_gs(w, "f64_native") as s:
        s.set_f(f0)
        s.step(steps)
        mg = s.moments()
        fg = s.get_f()
    assert np.max(np.abs(fg - fo)) <= 1e-12 * fo.max()
    for col in (1, 2, 3, 4, 5, 6):
        assert np.max(np.abs(mg[:, col] - mo[:, col])) <= 1e-11 * max(1.0, np.abs(mo[:, col]).max()), col


def test_gs_hmf_256_fp32_magnetisation_within_1e5():
    w = I.HMF_256
    f0 = I.initial_state(w)
    _, mo = O.run(grid_gs(w), f0, w.steps)
    with make_gs(w, "f32") as s:
        s.set_f(f0)
        s.step(w.steps)
        mg = s.moments()
    dM = np.abs(np.hypot(mg[:, 2], mg[:, 3]) - np.hypot(mo[:, 2], mo[:, 3]))
    assert dM.max() <= 1e-5
    assert np.max(np.abs(mg[:, 1] - 1.0)) <= 1e-5


def test_gs_and_fd_are_different_methods_of_similar_accuracy():
    """Tables 1-2: the two splines give norm and energy errors of one size (self-gravitating sheet)."""
    w = I.SHEET_4096.resized(256, 256)
    f0 = I.initial_state(w)
    drift = {}
    for spline in ("fd", "gs"):
        with V.Sim.from_workload(w, precision="f64_native") as s:
            s.spline = spline
            s.set_f(f0)
            s.step(100)
            m = s.moments()
            drift[spline] = (np.max(np.abs(m[:, 1] - m[0, 1])), np.max(np.abs(m[:, 6] / m[0, 6] - 1)))
            if spline == "fd":
                f_fd = s.get_f()
            else:
                f_gs = s.get_f()
    assert np.max(np.abs(f_fd - f_gs)) > 1e-8 * f_fd.max()        # not the same method
    for q in (0, 1):   # norm, energy: the same size within a factor of 20 (Table 1: up to 7x apart)
        assert 1 / 20 <= (drift["gs"][q] + 1e-15) / (drift["fd"][q] + 1e-15) <= 20, drift


def test_gs_api_rules():
    w = I.HMF_256.resized(128, 128)
    with V.Sim.from_workload(w, precision="fx64") as s:
        assert s.spline == "fd"
        with pytest.raises(V.VlasovError):
            s.spline = "gs"                    # IEEE FP64 or FP32 storage only
    with V.Sim.from_workload(I.HMF_256.resized(32, 128), precision="f64_native") as s:
        with pytest.raises(V.VlasovError):
            s.spline = "gs"                    # lines of 64 nodes or more
    with V.Sim.from_workload(w, precision="f32") as s:
        assert s.fused_x
        s.spline = "gs"
        assert s.spline == "gs" and not s.fused_x
        with pytest.raises(V.VlasovError):
            s.fused_x = True
        s.set_f(I.initial_state(w))
        s.step(3)
        s.spline = "fd"
        assert s.spline == "fd"
        s.step(2)
        assert s.moments().shape == (5, 8)
