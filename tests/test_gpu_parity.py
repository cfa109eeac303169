"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by element.

FP64 bar: one sweep agrees to rounding (1e-13 max|f| with IEEE FP64 filter arithmetic, "f64_native";
2e-14 max|f| with the integer/FP32 filter arithmetic of the default "f64" mode, whose error is about
2^-49 of 4 max|f| per sweep); 200 Strang steps of the 256^2 HMF workload agree to 1e-12 max f.  FP32
storage: one sweep agrees to 2e-6 max|f| (FP32 rounding of f and of the ten weights); the
magnetisation history agrees to |dM| <= 1e-5.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1206_3229_gb300 import inputs as I
from paper_1206_3229_gb300 import vlasov as V

pytestmark = pytest.mark.gpu

TOL_SWEEP = {"f64": 2e-14, "fx64": 2e-14, "f64_native": 1e-13, "f32": 2e-6}
PRECS = ["f64", "fx64", "f64_native", "f32"]
FP64_MODES = ["f64", "fx64", "f64_native"]


def grid_of(w: I.Workload) -> O.Grid:
    return O.Grid(w.model, w.nx, w.np, w.xmin, w.xmax, w.pmin, w.pmax, w.x_periodic, w.p_periodic,
                  w.dt, w.eps, w.G)


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def make(w, prec="f64"):
    return V.Sim.from_workload(w, precision=prec)


def rand_f(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, shape)


# ------------------------------------------------------------------------------------- sweeps
SWEEP_CASES = [
    # name, nx, np, x_periodic, p_periodic
    ("periodic_x_ragged", 200, 328, True, False),
    ("zero_x_ragged", 200, 328, False, False),
    ("periodic_p", 96, 144, True, True),
    ("tiny", 16, 16, True, False),
]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name,nx,np_,xper,pper", SWEEP_CASES)
def test_x_sweep_matches_oracle(prec, name, nx, np_, xper, pper):
    w = I.Workload(name, "free", nx, np_, -1.0, 1.0, -2.0, 2.0, xper, pper, 0.1, 1)
    rng = np.random.default_rng(nx + np_)
    f = rand_f((np_, nx), 1)
    for disp in (rng.uniform(-30, 30, np_), np.linspace(-3.3, 2.7, np_), np.round(rng.uniform(-9, 9, np_))):
        with make(w, prec) as s:
            s.set_f(f)
            s.substep(0, disp)
            got = s.get_f()
        want = O.advect_x(grid_of(w), f, disp)
        assert rel_err(got, want) <= TOL_SWEEP[prec], name


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name,nx,np_,xper,pper", SWEEP_CASES)
def test_p_sweep_matches_oracle(prec, name, nx, np_, xper, pper):
    w = I.Workload(name, "free", nx, np_, -1.0, 1.0, -2.0, 2.0, xper, pper, 0.1, 1)
    rng = np.random.default_rng(3 * nx + np_)
    f = rand_f((np_, nx), 2)
    x = np.arange(nx)
    cases = [
        4.0 * np.sin(2 * np.pi * x / nx) + 0.3,          # smooth, like a mean-field force (staged path)
        rng.uniform(-40, 40, nx),                          # large spread inside a tile (staged path)
        rng.uniform(-150, 150, nx),                        # spread beyond the staging buffer (direct path)
        np.full(nx, -1.0 * np_ - 7.5),                     # everything moved out of the grid
    ]
    for disp in cases:
        with make(w, prec) as s:
            s.set_f(f)
            s.substep(1, disp)
            got = s.get_f()
        want = O.advect_p(grid_of(w), f, disp)
        scale = max(np.max(np.abs(want)), np.max(np.abs(f)))
        assert np.max(np.abs(got - want)) <= TOL_SWEEP[prec] * scale, name


@pytest.mark.parametrize("prec", FP64_MODES)
def test_integer_free_streaming_is_exact_on_gpu(prec):
    """F = 0 and dp (dt/2)/dx = 1: three steps move row j by 6 (j - np/2) cells exactly."""
    nx, npp = 64, 32
    dx = 2 * math.pi / nx
    dp = 1.0 / 32
    w = I.Workload("free_int", "free", nx, npp, -math.pi, math.pi, -(npp // 2) * dp, (npp // 2) * dp,
                   True, False, 2 * dx / dp, 3)
    f0 = rand_f((npp, nx), 5)
    with make(w, prec) as s:
        s.set_f(f0)
        s.step(3)
        got = s.get_f()
    expect = np.stack([np.roll(f0[j], 6 * (j - npp // 2)) for j in range(npp)])
    if prec == "f64_native":
        # the foot fraction is exactly 0, so the filter is exactly (0, 0, 0, 0, 1, 0, ...)
        assert np.array_equal(got, expect)
        return
    # the split arithmetic rounds the FP32 part of every output to a multiple of 2^12 grid units,
    # 2^(Ef-49) (2^Ef >= 4 max f): the first sweep puts each value on that grid (at most half a step,
    # 2^(Ef-50), off), after which an integer shift reproduces it exactly (its low bits are zero, so
    # the FP32 conversion of its remainder is exact); plus the fixed-point upload (FX64, 2^(Ef-62)),
    # or the split of an IEEE double, which keeps 24 bits below 2^(Ef-31) (F64, 2^(Ef-55))
    Ef = math.frexp(float(np.abs(f0).max()))[1] + 2
    bound = 2.0 ** (Ef - 50) + (2.0 ** (Ef - 62) if prec == "fx64" else 2.0 ** (Ef - 55))
    err = float(np.max(np.abs(got - expect)))
    print(f"{prec}: integer free streaming, max |df| = {err:.3e} (bound {bound:.3e})")
    assert err <= bound


# ------------------------------------------------------------------------------------- density and forces
FORCE_CASES = [
    I.HMF_256.resized(128, 64),
    I.RING_2048.resized(256, 64),
    I.SHEET_4096.resized(256, 64),
]


@pytest.mark.parametrize("prec", FP64_MODES)
@pytest.mark.parametrize("w", FORCE_CASES, ids=lambda w: w.model)
def test_density_and_force_match_oracle(w, prec):
    f = I.initial_state(w)
    with make(w, prec) as s:
        s.set_f(f)
        rho, F = s.density_force()
    g = grid_of(w)
    rho_o = O.density(g, f)
    F_o = O.force(g, rho_o)
    assert rel_err(rho, rho_o) <= 1e-13
    assert rel_err(F, F_o) <= 1e-12


# ------------------------------------------------------------------------------------- full steps
@pytest.mark.parametrize("prec", FP64_MODES)
def test_hmf_256_fp64_200_steps_matches_oracle(prec):
    """The 256^2 HMF waterbag in FP64: max|df| <= 1e-12 max f after 200 steps; moments per step."""
    w = I.HMF_256
    f0 = I.initial_state(w)
    fo, mo = O.run(grid_of(w), f0, w.steps)
    with make(w, prec) as s:
        s.set_f(f0)
        s.step(w.steps)
        mg = s.moments()
        fg = s.get_f()
    assert np.max(np.abs(fg - fo)) <= 1e-12 * fo.max()
    assert mg.shape[0] == w.steps
    assert np.array_equal(mg[:, 7], np.arange(1, w.steps + 1))
    for col in (1, 2, 3, 4, 5, 6):   # mass, Mx, My, kinetic, potential, energy
        assert np.max(np.abs(mg[:, col] - mo[:, col])) <= 1e-12, col


@pytest.mark.parametrize("w,steps", [
    (I.RING_2048.resized(128, 128), 40),
    (I.SHEET_4096.resized(128, 256), 40),
    (I.HMF_4096_UNSTABLE.resized(128, 256), 40),
], ids=["ring", "sheet", "hmf_mode"])
@pytest.mark.parametrize("prec", FP64_MODES)
def test_models_fp64_steps_match_oracle(w, steps, prec):
    f0 = I.initial_state(w)
    fo, mo = O.run(grid_of(w), f0, steps)
    with make(w, prec) as s:
        s.set_f(f0)
        s.step(steps)
        mg = s.moments()
        fg = s.get_f()
    assert np.max(np.abs(fg - fo)) <= 1e-12 * fo.max()
    for col in (1, 2, 3, 4, 5, 6):
        assert np.max(np.abs(mg[:, col] - mo[:, col])) <= 1e-11 * max(1.0, np.abs(mo[:, col]).max()), col


def test_hmf_256_fp32_magnetisation_within_1e5():
    w = I.HMF_256
    f0 = I.initial_state(w)
    _, mo = O.run(grid_of(w), f0, w.steps)
    with make(w, "f32") as s:
        s.set_f(f0)
        s.step(w.steps)
        mg = s.moments()
    dM = np.abs(np.hypot(mg[:, 2], mg[:, 3]) - np.hypot(mo[:, 2], mo[:, 3]))
    assert dM.max() <= 1e-5
    assert np.max(np.abs(mg[:, 1] - 1.0)) <= 1e-5   # FP32 mass drift


def test_repeat_runs_are_bitwise_identical():
    """Fixed-order reductions: the same run twice gives the same bits."""
    w = I.HMF_256.resized(128, 128)
    f0 = I.initial_state(w)
    out = []
    for _ in range(2):
        with make(w) as s:
            s.set_f(f0)
            s.step(25)
            out.append((s.get_f(), s.moments()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_resume_from_downloaded_state_is_bitwise_identical():
    """Checkpoint/resume: get_f after k steps, set_f into a new handle, continue."""
    w = I.HMF_256.resized(128, 128)
    f0 = I.initial_state(w)
    with make(w) as s:
        s.set_f(f0)
        s.step(20)
        ref = s.get_f()
    with make(w) as a:
        a.set_f(f0)
        a.step(12)
        mid = a.get_f()
    with make(w) as b:
        b.set_f(mid)
        b.step(8)
        got = b.get_f()
    assert np.array_equal(ref, got)


# ------------------------------------------------------------------------------------- full-size samples
def test_full_size_hmf_4096_fp64_one_step_matches_oracle():
    """The 4096^2 HMF workload, in the launch shape the benchmark times: one step vs the oracle."""
    w = I.HMF_4096_UNSTABLE
    f0 = I.initial_state(w)
    O.set_threads(0)
    fo = O.step_parts(grid_of(w), f0)["out"]
    with make(w) as s:
        s.set_f(f0)
        s.step(1)
        fg = s.get_f()
    assert np.max(np.abs(fg - fo)) <= 1e-13 * fo.max()


def test_full_size_sheet_4096_fp64_one_step_matches_oracle():
    w = I.SHEET_4096
    f0 = I.initial_state(w)
    fo = O.step_parts(grid_of(w), f0)["out"]
    with make(w) as s:
        s.set_f(f0)
        s.step(1)
        fg = s.get_f()
    assert np.max(np.abs(fg - fo)) <= 1e-13 * fo.max()


def test_full_size_ring_2048_fp32_one_step_matches_oracle():
    w = I.RING_2048
    f0 = I.initial_state(w)
    fo = O.step_parts(grid_of(w), f0)["out"]
    with make(w, "f32") as s:
        s.set_f(f0)
        s.step(1)
        fg = s.get_f()
    assert np.max(np.abs(fg - fo)) <= 6e-6 * fo.max()


# ------------------------------------------------------------------------------------- physics on the GPU
def test_gpu_stationary_homogeneous_waterbag():
    w = I.Workload("hmf_stable", "hmf", 64, 128, -math.pi, math.pi, -2.0, 2.0, True, False, 0.05, 200,
                   init="mode", x0=math.pi, p0=math.sqrt(6 * (0.7 - 0.5)), mode_amp=0.0)
    f0 = I.initial_state(w)
    with make(w) as s:
        s.set_f(f0)
        s.step(200)
        f = s.get_f()
    assert np.max(np.abs(f - f0)) <= 1e-13 * f0.max()


def test_gpu_growth_rate_of_unstable_waterbag():
    w = I.Workload("hmf_unstable", "hmf", 64, 512, -math.pi, math.pi, -2.0, 2.0, True, False, 0.05, 420,
                   init="mode", x0=math.pi, p0=math.sqrt(6 * (0.55 - 0.5)), mode_amp=1e-6)
    f0 = I.initial_state(w)
    p = w.pmin + np.arange(w.np) * w.dp
    gamma_th = math.sqrt(0.5 - 3 * np.sum(f0 * (p ** 2)[:, None]) * w.dx * w.dp)
    with make(w) as s:
        s.set_f(f0)
        s.step(w.steps)
        m = s.moments()
    M = np.hypot(m[:, 2], m[:, 3])
    sel = (M > 1e-5) & (M < 1e-3)
    gamma = np.polyfit(m[sel, 0], np.log(M[sel]), 1)[0]
    assert abs(gamma - gamma_th) <= 0.05 * gamma_th


# ------------------------------------------------------------------------------------- API edge cases
def test_step_before_set_f_is_a_state_error():
    w = I.HMF_256.resized(64)
    with make(w) as s:
        with pytest.raises(V.VlasovError) as ei:
            s.step(1)
        assert ei.value.code == V.ESTATE


def test_zero_steps_and_empty_moment_history():
    w = I.HMF_256.resized(64)
    with make(w) as s:
        s.set_f(I.initial_state(w))
        s.step(0)
        assert s.moments().shape == (0, 8)
        s.step(3)
        assert s.moments().shape == (3, 8)
        assert s.moments().shape == (0, 8)


def test_moment_ring_keeps_the_latest_records():
    w = I.HMF_256.resized(16, 16)
    with make(w) as s:
        s.set_f(I.initial_state(w))
        s.step(4096 + 10)
        m = s.moments(max_records=8192)
    assert m.shape[0] == 4096 and m[-1, 7] == 4106 and m[0, 7] == 11


def test_device_pointer_round_trip():
    torch = pytest.importorskip("torch")
    w = I.HMF_256.resized(64)
    f0 = I.initial_state(w)
    src = torch.from_numpy(f0).cuda()
    dst = torch.empty_like(src)
    torch.cuda.synchronize()
    with make(w, "f32") as s:
        s.set_f_device(src.data_ptr())
        s.get_f_device(dst.data_ptr())
        s.sync()
    assert np.max(np.abs(dst.cpu().numpy() - f0)) <= 1e-7 * f0.max()


# ------------------------------------------------------------------------------------- maximum sizes
MAX_NX = {"f64": 8192, "fx64": 8192, "f64_native": 8192, "f32": 8192}


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("xper", [True, False])
def test_longest_rows_match_oracle(prec, xper):
    """The longest row each storage mode takes (a whole row per thread block): x and p sweeps at
    that Nx against the oracle, and one cell more is refused at creation."""
    nx, np_ = MAX_NX[prec], 72
    w = I.Workload("longest", "free", nx, np_, -1.0, 1.0, -2.0, 2.0, xper, False, 0.1, 1)
    rng = np.random.default_rng(nx + int(xper))
    f = rng.uniform(0.0, 1.0, (np_, nx))
    xdisp = rng.uniform(-40, 40, np_)
    pdisp = 6.0 * np.sin(2 * np.pi * np.arange(nx) / nx) - 0.4
    with make(w, prec) as s:
        s.set_f(f)
        s.substep(0, xdisp)
        gx = s.get_f()
        s.set_f(f)
        s.substep(1, pdisp)
        gp = s.get_f()
    assert rel_err(gx, O.advect_x(grid_of(w), f, xdisp)) <= TOL_SWEEP[prec]
    want = O.advect_p(grid_of(w), f, pdisp)
    assert np.max(np.abs(gp - want)) <= TOL_SWEEP[prec] * max(np.abs(want).max(), np.abs(f).max())
    with pytest.raises(V.VlasovError):
        make(w.resized(nx + 8, np_), prec)


@pytest.mark.parametrize("prec", FP64_MODES)
def test_hmf_rows_of_8192_cells_match_oracle(prec):
    """8-byte rows longer than 4096 cells (x-shift CTAs of 512 threads; the fused x-shifts, which hold
    rows of at most 4096 cells, are off): 20 steps of the HMF waterbag at 8192 x 96 against the
    oracle, f to 1e-12 max f and every step's moments to 1e-12."""
    w = I.HMF_256.resized(8192, 96, steps=20)
    f0 = I.initial_state(w)
    fo, mo = O.run(grid_of(w), f0, w.steps)
    with make(w, prec) as s:
        assert not s.fused_x
        s.set_f(f0)
        s.step(w.steps)
        mg = s.moments()
        fg = s.get_f()
    assert np.max(np.abs(fg - fo)) <= 1e-12 * fo.max()
    for col in (1, 2, 3, 4, 5, 6):
        assert np.max(np.abs(mg[:, col] - mo[:, col])) <= 1e-12, col
