"""Fused x-shifts: the second x half-shift of step n and the first of step n+1 (Sec. 3, steps four and
one) run as one launch that keeps the row between them in shared memory.  The arithmetic of each pass
is that of the separate x-shift launches and every cross-CTA sum is exact, so a fused run must give
the same bits as an unfused one: f, and every moment record.  Also checked here: the full-size
4096^2 HMF workload in the launch configuration the benchmark times (FX64, fused, several steps)
against the oracle, and the launch accounting.

With FP32 or BF16 storage the fused launch runs the same per-pass arithmetic, but the per-CTA column
and kinetic sums are FP32 sums over that launch's own row partition: free streaming (no force) must
still give the same bits, a self-consistent run the same state to within the rounding of those sums."""
import numpy as np
import pytest

import oracle as O
from paper_1206_3229_gb300 import inputs as I
from paper_1206_3229_gb300 import vlasov as V

pytestmark = pytest.mark.gpu


def grid_of(w: I.Workload) -> O.Grid:
    return O.Grid(w.model, w.nx, w.np, w.xmin, w.xmax, w.pmin, w.pmax, w.x_periodic, w.p_periodic,
                  w.dt, w.eps, w.G)


def run(w, f0, steps, fused, calls=None, precision="fx64"):
    with V.Sim.from_workload(w, precision=precision) as s:
        s.fused_x = fused
        s.set_f(f0)
        for n in (calls or [steps]):
            s.step(n)
        return s.get_f(), s.moments()


@pytest.mark.parametrize("w", [
    I.HMF_256.resized(256, 256),
    I.HMF_4096_UNSTABLE.resized(512, 384),
    I.RING_2048.resized(128, 128),
    I.SHEET_4096.resized(128, 256),
    I.HMF_256.resized(320, 328),          # ragged: 40 active threads of 64, boxes of 40 lines
], ids=["hmf", "hmf_mode", "ring", "sheet", "ragged"])
def test_fused_run_is_bitwise_the_unfused_run(w):
    f0 = I.initial_state(w)
    fa, ma = run(w, f0, 30, fused=False)
    fb, mb = run(w, f0, 30, fused=True)
    assert np.array_equal(fa, fb)
    assert ma.shape == mb.shape == (30, 8)
    assert np.array_equal(ma, mb)


@pytest.mark.parametrize("w", [
    # free streaming on a zero-outside x axis with |displacement| up to 64 cells: 80-element halos,
    # two 640-byte groups of zero lines before each staged row
    I.Workload("free_far", "free", 256, 128, -8.0, 8.0, -4.0, 4.0, False, False, 2.0, 4),
    I.HMF_256.resized(64, 16),            # smallest fused grid: one 8-line box per row, 16 rows
], ids=["zero_x_far_shift", "tiny"])
def test_fused_edge_cases_are_bitwise_the_unfused_run(w):
    x = w.xmin + w.dx * np.arange(w.nx)
    p = w.pmin + w.dp * np.arange(w.np)
    f0 = np.exp(-0.5 * (x[None, :] / 1.5) ** 2 - (p[:, None] / 1.2) ** 2)   # smooth, ~0 at the edges
    fa, ma = run(w, f0, 4, fused=False)
    fb, mb = run(w, f0, 4, fused=True)
    assert np.array_equal(fa, fb) and np.array_equal(ma, mb)
    assert np.abs(fa).max() > 0.1


def test_split_calls_give_the_same_bits():
    """Steps enqueued as 1 + 2 + 7 calls (head/tail pieces at every boundary) = one call of 10."""
    w = I.HMF_256.resized(128, 128)
    f0 = I.initial_state(w)
    fa, ma = run(w, f0, 10, fused=True)
    fb, mb = run(w, f0, 10, fused=True, calls=[1, 2, 7])
    assert np.array_equal(fa, fb) and np.array_equal(ma, mb)


def test_full_size_hmf_4096_fx64_fused_steps_match_oracle():
    """The 4096^2 HMF workload as the benchmark runs it (FX64, fused x-shifts, one call of 3 steps)."""
    w = I.HMF_4096_UNSTABLE
    f0 = I.initial_state(w)
    O.set_threads(0)
    steps = 3
    fo, mo = O.run(grid_of(w), f0, steps)
    with V.Sim.from_workload(w, precision="fx64") as s:
        assert s.fused_x
        s.set_f(f0)
        s.step(steps)
        fg = s.get_f()
        mg = s.moments()
    assert np.max(np.abs(fg - fo)) <= 1e-13 * steps * fo.max()
    for col in (1, 2, 3, 4, 5, 6):
        assert np.max(np.abs(mg[:, col] - mo[:, col])) <= 1e-12 * max(1.0, np.abs(mo[:, col]).max()), col


def test_launch_accounting_and_timed_slots():
    w = I.HMF_256.resized(128, 128)
    with V.Sim.from_workload(w, precision="fx64") as s:
        s.set_f(I.initial_state(w))
        assert s.fused_x
        L = s.kernels_per_step()
        assert L == 4 and len(s.slot_names()) == L
        # head: x-shift, filters, p-shift; n-1 mids; tail: x-shift, moments
        assert s.launches(1) == 5 and s.launches(10) == 3 + 9 * L + 2
        ms = s.step_timed(3)
        assert ms.shape == (L,) and np.all(ms > 0)
        s.fused_x = False
        assert s.kernels_per_step() == 5 and s.launches(10) == 50
    with V.Sim.from_workload(w, precision="f64") as s:
        assert not s.fused_x
        with pytest.raises(V.VlasovError):
            s.fused_x = True


def test_launches_with_filters_formed_in_other_launches():
    """FP32 HMF: the p-shift forms its filters itself (fused x-shifts, moment record, p-shift); the ring
    with the fixed-point force: its force launch writes the filters (fused x-shifts, merged reductions,
    convolutions, p-shift).  The timed slots match the launches."""
    w = I.HMF_256.resized(128, 128)
    for prec in ("f32", "bf16"):
        with V.Sim.from_workload(w, precision=prec) as s:
            s.set_f(I.initial_state(w))
            L = s.kernels_per_step()
            assert L == 3 and s.slot_names() == ["xshift_fused", "reduce_moments", "pshift_step3"]
            # head: x-shift, p-shift; n-1 mids; tail: x-shift, moments
            assert s.launches(1) == 4 and s.launches(10) == 2 + 9 * L + 2
            assert s.step_timed(3).shape == (L,)
            s.fused_x = False
            assert s.kernels_per_step() == 4 and len(s.slot_names()) == 4 and s.launches(10) == 40
    r = I.RING_2048.resized(128, 128)
    for prec in ("fx64", "f32"):
        with V.Sim.from_workload(r, precision=prec) as s:
            s.set_f(I.initial_state(r))
            assert s.ring_method == "fixed"
            L = s.kernels_per_step()
            assert L == 4 and len(s.slot_names()) == L
            assert s.step_timed(3).shape == (L,)
            s.ring_method = "direct"   # the filters get a launch of their own again
            assert s.kernels_per_step() == L + 3 and len(s.slot_names()) == L + 3


FREE_PERIODIC = I.Workload("free_periodic", "free", 512, 256, -np.pi, np.pi, -4.0, 4.0, True, False, 0.05, 4)
FREE_ZERO = I.Workload("free_zero", "free", 256, 128, -8.0, 8.0, -4.0, 4.0, False, False, 2.0, 4)


def smooth_f0(w):
    x = w.xmin + w.dx * np.arange(w.nx)
    p = w.pmin + w.dp * np.arange(w.np)
    return np.exp(-0.5 * (x[None, :] / 1.5) ** 2 - (p[:, None] / 1.2) ** 2)


@pytest.mark.parametrize("precision", ["f32", "bf16"])
@pytest.mark.parametrize("w", [FREE_PERIODIC, FREE_ZERO], ids=["periodic", "zero_outside"])
def test_fp32_class_fused_free_streaming_is_bitwise(w, precision):
    f0 = smooth_f0(w)
    fa, ma = run(w, f0, 12, fused=False, precision=precision)
    fb, mb = run(w, f0, 12, fused=True, precision=precision)
    assert np.array_equal(fa, fb)
    assert np.abs(fa).max() > 0.1
    # mass: per-CTA FP32 column sums of another row partition, then exact fixed-point totals
    np.testing.assert_allclose(mb[:, 1], ma[:, 1], rtol=1e-6, atol=0)


# (tolerance on f relative to max f, tolerance on the mass, on the other moments relative to their scale)
FP32_CLASS_TOL = {"f32": (1e-5, 1e-6, 1e-5), "bf16": (5e-2, 1e-3, 2e-2)}


@pytest.mark.parametrize("precision", ["f32", "bf16"])
@pytest.mark.parametrize("w", [
    I.HMF_256.resized(256, 256),
    I.RING_2048.resized(128, 128),
    I.SHEET_4096.resized(128, 256),
    I.HMF_256.resized(320, 328),
], ids=["hmf", "ring", "sheet", "ragged"])
def test_fp32_class_fused_run_matches_unfused(w, precision):
    f0 = I.initial_state(w)
    steps = 30
    fa, ma = run(w, f0, steps, fused=False, precision=precision)
    fb, mb = run(w, f0, steps, fused=True, precision=precision)
    tf, tm, to = FP32_CLASS_TOL[precision]
    assert np.max(np.abs(fa - fb)) <= tf * np.abs(fa).max()
    assert ma.shape == mb.shape == (steps, 8)
    assert np.array_equal(ma[:, 0], mb[:, 0]) and np.array_equal(ma[:, 7], mb[:, 7])   # t, step
    assert np.max(np.abs(ma[:, 1] - mb[:, 1])) <= tm * np.abs(ma[:, 1]).max()
    for col in (2, 3, 4, 5, 6):
        scale = max(np.abs(ma[:, col]).max(), 1e-3 * np.abs(ma[:, 4]).max())
        assert np.max(np.abs(ma[:, col] - mb[:, col])) <= to * scale, col


@pytest.mark.parametrize("precision", ["f32", "bf16"])
def test_fp32_class_fused_defaults_and_accounting(precision):
    w = I.HMF_256.resized(128, 128)
    with V.Sim.from_workload(w, precision=precision) as s:
        s.set_f(I.initial_state(w))
        assert s.fused_x                            # on by default for FP32-class storage
        s.fused_x = True
        L = s.kernels_per_step()
        assert len(s.slot_names()) == L
        assert s.launches(10) == s.launches(2) + 8 * L   # head + n-1 mids + tail
        ms = s.step_timed(3)
        assert ms.shape == (L,) and np.all(ms > 0)
    w = I.SHEET_4096.resized(128, 256)
    with V.Sim.from_workload(w, precision=precision) as s:
        assert s.fused_x
        s.fused_x = False
        assert not s.fused_x
    if precision == "f32":   # (BF16 grids are limited to Nx <= 4096 altogether)
        with V.Sim.from_workload(I.HMF_256.resized(4104, 16), precision=precision) as s:
            assert not s.fused_x                   # rows longer than 4096 cells: separate x-shifts
            with pytest.raises(V.VlasovError):
                s.fused_x = True


def test_full_size_hmf_4096_fp32_fused_steps_match_oracle():
    """The 4096^2 HMF workload with FP32 storage (fused x-shifts on by default), one call of 3 steps:
    f within the FP32 sweep bar (2e-6 max f per sweep, 9 sweeps), mass and magnetisation to 1e-6."""
    w = I.HMF_4096_UNSTABLE
    f0 = I.initial_state(w)
    O.set_threads(0)
    steps = 3
    fo, mo = O.run(grid_of(w), f0, steps)
    with V.Sim.from_workload(w, precision="f32") as s:
        assert s.fused_x
        s.set_f(f0)
        s.step(steps)
        fg = s.get_f()
        mg = s.moments()
    assert np.max(np.abs(fg - fo)) <= 2e-6 * 3 * steps * fo.max()
    assert np.max(np.abs(mg[:, 1] - mo[:, 1])) <= 1e-6
    assert np.max(np.abs(np.hypot(mg[:, 2], mg[:, 3]) - np.hypot(mo[:, 2], mo[:, 3]))) <= 1e-6


@pytest.mark.parametrize("precision", ["fx64", "f64_native", "f32"])
def test_graph_runs_give_the_bits_of_single_steps(precision):
    """vlasov_step(70) launches graphs of 2^L steps (fused middles or whole steps: 32 + 32 + 4 + 2
    ...); the same 70 steps as 70 calls of one step give the same bits, f and every moment record."""
    w = I.HMF_256.resized(128, 128)
    f0 = I.initial_state(w)
    fused = precision == "fx64"   # FX64: fused middles (= separate launches bitwise); else whole steps
    fa, ma = run(w, f0, 70, fused=fused, precision=precision)
    fb, mb = run(w, f0, 70, fused=fused, calls=[1] * 70, precision=precision)
    assert np.array_equal(fa, fb) and np.array_equal(ma, mb)
    assert ma.shape == (70, 8)
