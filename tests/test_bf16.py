"""BF16 storage experiment (VLASOV_BF16): f held in bfloat16 (8 significant bits), interpolated in
FP32, with FP64-accurate displacements and moment sums as in the FP32 path.  Sweeps are checked
against the FP64 oracle applied to the stored (rounded) input, so that only the rounding of the
output and FP32 arithmetic remain; the 200-step HMF run reports how far |M(t)| drifts from FP64."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1206_3229_gb300 import inputs as I
from paper_1206_3229_gb300 import vlasov as V

pytestmark = pytest.mark.gpu

ULP = 2.0 ** -7   # spacing of bf16 values in [1, 2): rounding to nearest moves a value by <= 2^-8 of it


def grid_of(w):
    return O.Grid(w.model, w.nx, w.np, w.xmin, w.xmax, w.pmin, w.pmax, w.x_periodic, w.p_periodic,
                  w.dt, w.eps, w.G)


def bf16_round(f):
    """Round to nearest even bf16 from FP32 bit patterns (exact for inputs that are FP32 values)."""
    u = np.asarray(f, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def test_upload_rounds_to_nearest_even():
    w = I.HMF_256.resized(64, 32)
    rng = np.random.default_rng(11)
    f = rng.uniform(-1.0, 1.0, (32, 64)).astype(np.float32).astype(np.float64)
    f[0, :4] = [1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 0.0, -2.5]   # ties go to even; exact values stay
    with V.Sim.from_workload(w, precision="bf16") as s:
        s.set_f(f)
        got = s.get_f()
    assert np.array_equal(got, bf16_round(f))
    assert got[0, 0] == 1.0 and got[0, 1] == 1.0 + 4 * 2 ** -8 and got[0, 3] == -2.5


SWEEP_CASES = [("periodic_x_ragged", 200, 328, True, False), ("zero_x_ragged", 200, 328, False, False),
               ("periodic_p", 96, 144, True, True), ("tiny", 16, 16, True, False)]


@pytest.mark.parametrize("name,nx,np_,xper,pper", SWEEP_CASES)
def test_sweeps_match_the_oracle_on_the_stored_input(name, nx, np_, xper, pper):
    w = I.Workload(name, "free", nx, np_, -1.0, 1.0, -2.0, 2.0, xper, pper, 0.1, 1)
    rng = np.random.default_rng(nx + 7 * np_)
    f = rng.uniform(0.0, 1.0, (np_, nx))
    cases = [(0, rng.uniform(-30, 30, np_)), (0, np.linspace(-3.3, 2.7, np_)),
             (1, 4.0 * np.sin(2 * np.pi * np.arange(nx) / nx) + 0.3), (1, rng.uniform(-150, 150, nx))]
    for axis, disp in cases:
        with V.Sim.from_workload(w, precision="bf16") as s:
            s.set_f(f)
            f_in = s.get_f()
            s.substep(axis, disp)
            got = s.get_f()
        g = grid_of(w)
        want = O.advect_x(g, f_in, disp) if axis == 0 else O.advect_p(g, f_in, disp)
        scale = max(np.abs(want).max(), np.abs(f_in).max())
        assert np.max(np.abs(got - want)) <= 0.5 * ULP * 1.02 * scale, (name, axis)


def test_integer_free_streaming_is_exact():
    nx, npp = 64, 32
    dx = 2 * math.pi / nx
    dp = 1.0 / 32
    w = I.Workload("free_int", "free", nx, npp, -math.pi, math.pi, -(npp // 2) * dp, (npp // 2) * dp,
                   True, False, 2 * dx / dp, 3)
    f0 = bf16_round(np.random.default_rng(5).uniform(0, 1, (npp, nx)).astype(np.float32))
    with V.Sim.from_workload(w, precision="bf16") as s:
        s.set_f(f0)
        s.step(3)
        got = s.get_f()
    assert np.array_equal(got, np.stack([np.roll(f0[j], 6 * (j - npp // 2)) for j in range(npp)]))


def test_hmf_256_200_steps_magnetisation_drift_from_fp64():
    """The experiment's number: |dM(t)| of bf16 storage against the FP64 oracle over 200 steps of the
    256^2 HMF waterbag (the FP32 path holds 1e-5 here); mass stays within bf16 rounding."""
    w = I.HMF_256
    f0 = I.initial_state(w)
    _, mo = O.run(grid_of(w), f0, w.steps)
    with V.Sim.from_workload(w, precision="bf16") as s:
        s.set_f(f0)
        s.step(w.steps)
        mg = s.moments()
        S, Q = s.casimirs()
        f = s.get_f()
    dM = np.abs(np.hypot(mg[:, 2], mg[:, 3]) - np.hypot(mo[:, 2], mo[:, 3]))
    print(f"bf16 storage, HMF 256^2, 200 steps: max |dM| = {dM.max():.3e}, "
          f"max |d mass| = {np.abs(mg[:, 1] - mo[:, 1]).max():.3e}")
    assert dM.max() <= 2e-2
    assert np.abs(mg[:, 1] - 1.0).max() <= 2e-2
    g = grid_of(w)
    assert S == pytest.approx(O.entropy(g, f), rel=1e-13)
    assert Q == pytest.approx(O.moments(g, f)["l2"], rel=1e-13)
