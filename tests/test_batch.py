"""Batched form (many simulations per launch) and the continuous-batching serving loop (GPU).

* A simulation gives bit-identical results alone in a batch and in a mix of other models, sizes
  and admission times (its own fixed CTA-to-row mapping; order-free integer moment sums).
* It agrees with the single-grid FP32 path and with the FP64 oracle within the FP32 tolerance.
* The device-side initial state equals the shared input generator's.
* The serving loop admits by arrival time, slots and memory, and reproduces the alone-results.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1206_3229_gb300 import inputs as I
from paper_1206_3229_gb300 import vlasov as V

pytestmark = pytest.mark.gpu

GB = 1 << 30


def grid_of(w):
    return O.Grid(w.model, w.nx, w.np, w.xmin, w.xmax, w.pmin, w.pmax, w.x_periodic, w.p_periodic, w.dt, w.eps, w.G)


HMF_R = I.HMF_256
MIX = [
    I.RING_2048.resized(128, 128),
    I.SHEET_4096.resized(256, 256),
    I.HMF_4096_UNSTABLE.resized(512, 256),
    I.RING_2048.resized(256, 192),
]


def run_alone(w, steps, slots=4):
    with V.Batch(slots, 512, GB) as b:
        k = b.admit(V.request_from_workload(w, steps))
        b.step(steps + 3)
        assert b.steps_done(k) == steps
        return b.get(k, w.nx, w.np)


def test_alone_equals_in_mix_bitwise():
    steps = 30
    f_a, m_a = run_alone(HMF_R, steps)
    with V.Batch(8, 512, 2 * GB) as b:
        others = [b.admit(V.request_from_workload(w, 7 + 5 * q)) for q, w in enumerate(MIX[:3])]
        b.step(5)
        k = b.admit(V.request_from_workload(HMF_R, steps))
        b.step(2)
        late = b.admit(V.request_from_workload(MIX[3], 12))
        b.step(steps + 5)
        f_b, m_b = b.get(k, HMF_R.nx, HMF_R.np)
        assert b.steps_done(k) == steps and b.steps_done(late) == 12
        assert all(b.steps_done(o) == 7 + 5 * q for q, o in enumerate(others))
    assert np.array_equal(f_a, f_b)
    assert np.array_equal(m_a, m_b)
    assert m_a.shape == (steps, 8)


def test_batch_matches_single_grid_f32_path():
    w = HMF_R
    steps = 40
    f0 = I.initial_state(w)
    with V.Batch(2, 256, GB) as b:
        k = b.admit(V.request_from_workload(w, steps), f0)
        b.step(steps)
        fb, mb = b.get(k, w.nx, w.np)
    with V.Sim.from_workload(w, precision="f32") as s:
        s.set_f(f0)
        s.step(steps)
        ms = s.moments()
        fs = s.get_f()
    assert np.max(np.abs(fb - fs)) <= 1e-5 * fs.max()
    assert np.max(np.abs(np.hypot(mb[:, 2], mb[:, 3]) - np.hypot(ms[:, 2], ms[:, 3]))) <= 1e-6


def test_batch_fp32_against_oracle_magnetisation():
    w = HMF_R
    steps = 100
    f0 = I.initial_state(w)
    _, mo = O.run(grid_of(w), f0, steps)
    with V.Batch(2, 256, GB) as b:
        k = b.admit(V.request_from_workload(w, steps), f0)
        b.step(steps)
        _, mb = b.get(k, w.nx, w.np)
    dM = np.abs(np.hypot(mb[:, 2], mb[:, 3]) - np.hypot(mo[:, 2], mo[:, 3]))
    assert dM.max() <= 1e-5
    assert np.max(np.abs(mb[:, 1] - 1.0)) <= 1e-5


@pytest.mark.parametrize("w", [I.HMF_256, I.RING_2048.resized(256, 128), I.SHEET_4096.resized(256, 256),
                               I.HMF_4096_UNSTABLE.resized(128, 256)], ids=lambda w: w.name)
def test_device_initial_state_matches_input_generator(w):
    with V.Batch(1, 256, GB) as b:
        k = b.admit(V.request_from_workload(w, 0))
        f, _ = b.get(k, w.nx, w.np)
    ref = I.initial_state(w)
    assert np.max(np.abs(f - ref)) <= 2e-6 * ref.max()


def test_serve_stream_reproduces_alone_results():
    rng = np.random.default_rng(11)
    pool = [I.HMF_256, I.RING_2048.resized(128, 128), I.SHEET_4096.resized(256, 256),
            I.HMF_4096_UNSTABLE.resized(256, 256)]
    reqs, ws = [], []
    t = 0.0
    for q in range(10):
        w = pool[q % len(pool)]
        steps = int(rng.integers(5, 25))
        t += float(rng.exponential(0.01))
        reqs.append(V.request_from_workload(w, steps, arrival_s=t))
        ws.append((w, steps))
    budget = 3 * max(V.batch_footprint(r) for r in reqs)
    results, makespan = V.serve(reqs, slots=4, mem_budget_bytes=budget, max_n=256)
    assert makespan > 0
    for (w, steps), r in zip(ws, results):
        assert r.status == 0 and r.steps == steps
        assert r.admit_s >= r.arrival_s - 1e-6 and r.done_s >= r.admit_s - 1e-3
        _, m = run_alone(w, steps)
        assert V.moments_row(r.last) == list(m[-1])
        assert V.moments_row(r.first) == list(m[0])


def test_serve_admission_waits_for_memory():
    big = V.request_from_workload(I.HMF_4096_UNSTABLE.resized(512, 512), 20, arrival_s=0.0)
    big2 = V.request_from_workload(I.HMF_4096_UNSTABLE.resized(512, 512), 20, arrival_s=0.0)
    budget = int(1.5 * V.batch_footprint(big))
    results, _ = V.serve([big, big2], slots=4, mem_budget_bytes=budget, max_n=512)
    a, c = results
    assert a.status == 0 and c.status == 0
    first, second = (a, c) if a.admit_s <= c.admit_s else (c, a)
    assert second.admit_s >= first.done_s - 1e-3   # only one fits at a time


def test_batch_rejects_bad_requests():
    with V.Batch(1, 256, GB) as b:
        bad = V.request_from_workload(I.HMF_256.resized(512), 1)
        with pytest.raises(V.VlasovError) as ei:
            b.admit(bad)
        assert ei.value.code == V.EINVAL
        k = b.admit(V.request_from_workload(I.HMF_256, 1))
        with pytest.raises(V.VlasovError) as ei:
            b.admit(V.request_from_workload(I.HMF_256, 1))
        assert ei.value.code == V.ESTATE
        b.release(k)
        b.admit(V.request_from_workload(I.HMF_256, 1))


# ------------------------------------------------------------------------------ FX64 (FP64-accurate) slots
FX_CASES = [I.HMF_256, I.RING_2048.resized(128, 128), I.SHEET_4096.resized(256, 256),
            I.HMF_4096_UNSTABLE.resized(256, 256)]


@pytest.mark.parametrize("w", FX_CASES, ids=lambda w: w.name)
def test_fx64_batch_is_bitwise_the_single_grid_fx64_path(w):
    """Same sweep kernels, same fixed-point bound from the same f0: identical f for ring and sheet,
    and identical moment records (every sum, the kinetic one included, is an exact fixed-point sum,
    whatever the CTA partition).  HMF: the single-grid path forms Mx, My from per-CTA partials with
    50-bit cos/sin weights, the batch from per-column totals with 62-bit weights, so the force
    differs in its last bits and f agrees to rounding."""
    steps = 25
    f0 = I.initial_state(w)
    with V.Batch(2, 512, GB, precision="fx64") as b:
        k = b.admit(V.request_from_workload(w, steps), f0)
        b.step(steps)
        fb, mb = b.get(k, w.nx, w.np)
    with V.Sim.from_workload(w, precision="fx64") as s:
        s.set_f(f0)
        s.step(steps)
        ms = s.moments()
        fs = s.get_f()
    if w.model == "hmf":
        assert np.max(np.abs(fb - fs)) <= 1e-13 * fs.max()
        for col in (1, 2, 3, 4, 5):
            assert np.max(np.abs(mb[:, col] - ms[:, col])) <= 1e-13, col
        return
    assert np.array_equal(fb, fs)
    for col in (1, 2, 3, 4, 5, 6):   # mass, Mx, My, kinetic, potential, energy
        assert np.array_equal(mb[:, col], ms[:, col]), col


def test_fx64_batch_alone_equals_in_mix_bitwise():
    steps = 20
    f_a = None
    with V.Batch(2, 512, GB, precision="fx64") as b:
        k = b.admit(V.request_from_workload(HMF_R, steps))
        b.step(steps + 2)
        f_a, m_a = b.get(k, HMF_R.nx, HMF_R.np)
    with V.Batch(6, 512, 2 * GB, precision="fx64") as b:
        others = [b.admit(V.request_from_workload(w, 5 + 4 * q)) for q, w in enumerate(MIX[:3])]
        b.step(3)
        k = b.admit(V.request_from_workload(HMF_R, steps))
        b.step(1)
        b.admit(V.request_from_workload(MIX[3], 9))
        b.step(steps + 4)
        f_b, m_b = b.get(k, HMF_R.nx, HMF_R.np)
        assert b.steps_done(k) == steps
        assert all(b.steps_done(o) == 5 + 4 * q for q, o in enumerate(others))
    assert np.array_equal(f_a, f_b)
    assert np.array_equal(m_a, m_b)


def test_fx64_batch_against_oracle_fp64_tolerance():
    """The FX64 batched form meets the FP64 parity bar: 100 HMF steps at 256^2."""
    w = HMF_R
    steps = 100
    f0 = I.initial_state(w)
    fo, mo = O.run(grid_of(w), f0, steps)
    with V.Batch(1, 256, GB, precision="fx64") as b:
        k = b.admit(V.request_from_workload(w, steps), f0)
        b.step(steps)
        fb, mb = b.get(k, w.nx, w.np)
    assert np.max(np.abs(fb - fo)) <= 1e-12 * fo.max()
    assert np.max(np.abs(np.hypot(mb[:, 2], mb[:, 3]) - np.hypot(mo[:, 2], mo[:, 3]))) <= 1e-12


@pytest.mark.parametrize("w", [I.HMF_256, I.SHEET_4096.resized(256, 256), I.HMF_4096_UNSTABLE.resized(128, 256)],
                         ids=lambda w: w.name)
def test_fx64_device_initial_state_matches_input_generator(w):
    with V.Batch(1, 256, GB, precision="fx64") as b:
        k = b.admit(V.request_from_workload(w, 0))
        f, _ = b.get(k, w.nx, w.np)
    ref = I.initial_state(w)
    assert np.max(np.abs(f - ref)) <= 1e-14 * ref.max()


def test_fx64_serve_results_equal_single_grid_moments():
    pool = [I.HMF_256, I.RING_2048.resized(128, 128), I.SHEET_4096.resized(256, 256)]
    reqs, ws = [], []
    for q in range(6):
        w = pool[q % len(pool)]
        steps = 6 + 3 * q
        reqs.append(V.request_from_workload(w, steps, arrival_s=0.002 * q))
        ws.append((w, steps))
    budget = 3 * max(V.batch_footprint(r, "fx64") for r in reqs)
    results, _ = V.serve(reqs, slots=3, mem_budget_bytes=budget, max_n=256, precision="fx64")
    for (w, steps), r in zip(ws, results):
        assert r.status == 0 and r.steps == steps
        with V.Batch(1, 256, GB, precision="fx64") as b:
            k = b.admit(V.request_from_workload(w, steps))
            b.step(steps)
            _, m = b.get(k, w.nx, w.np)
        assert V.moments_row(r.last) == list(m[-1])


def test_serve_rejects_unknown_precision():
    req = V.request_from_workload(I.HMF_256.resized(64), 3)
    with pytest.raises(ValueError):
        V.serve([req], slots=1, mem_budget_bytes=GB, precision="f64")


def test_batch_rejects_other_precisions():
    with pytest.raises(ValueError):
        V.Batch(1, 256, GB, precision="f64")


# ------------------------------------------------------------------------------------- launch shape
def run_shaped(prec, shape, ws, steps):
    out = []
    with V.Batch(4, 512, GB, precision=prec, shape=shape) as b:
        assert b.shape == shape
        ks = [b.admit(V.request_from_workload(w, steps)) for w in ws]
        b.step(steps + 2)
        for k, w in zip(ks, ws):
            out.append(b.get(k, w.nx, w.np))
    return out


SHAPE_MIX = [HMF_R, I.RING_2048.resized(128, 128), I.SHEET_4096.resized(256, 128)]


def test_fx64_batch_results_do_not_depend_on_the_launch_shape():
    """Exact fixed-point sums (column sums, HMF numbers, int128 kinetic partials): f and every moment
    record are the same bits for the smallest and the largest candidate shape."""
    a = run_shaped("fx64", (8, 4), SHAPE_MIX, 12)
    b = run_shaped("fx64", (32, 16), SHAPE_MIX, 12)
    for (fa, ma), (fb, mb) in zip(a, b):
        assert np.array_equal(fa, fb) and np.array_equal(ma, mb)


def test_f32_batch_depends_on_the_launch_shape_at_rounding_level_only():
    """FP32 slots: each CTA's FP64 column sums are rounded to fixed point before the exact sum over
    CTAs, so another row partition moves the density, hence the force, in its last bits, and f then
    differs by FP32 roundings (one ulp here and there); the moments of such f differ by about 1e-8,
    three orders below the FP32 path's |dM| <= 1e-5 bar."""
    a = run_shaped("f32", (8, 4), SHAPE_MIX, 12)
    b = run_shaped("f32", (32, 16), SHAPE_MIX, 12)
    for (fa, ma), (fb, mb) in zip(a, b):
        assert np.max(np.abs(fa - fb)) <= 1e-6 * np.abs(fa).max()
        assert np.max(np.abs(ma[:, 1:7] - mb[:, 1:7])) <= 1e-7 * max(1.0, np.abs(ma[:, 1:7]).max())


@pytest.mark.parametrize("prec", ["f32", "fx64"])
def test_autotune_picks_the_fastest_candidate_and_later_batches_use_it(prec):
    best, ms = V.batch_autotune(256, prec)
    assert best in V.AUTOTUNE_CANDIDATES
    ran = {c: t for c, t in ms.items() if t > 0}
    assert len(ran) == len(V.AUTOTUNE_CANDIDATES) and ran[best] == min(ran.values())
    with V.Batch(2, 256, GB // 4, precision=prec) as b:
        assert b.shape == best
    with V.Batch(2, 128, GB // 4, precision=prec) as b:   # another max_n keeps the default
        assert b.shape == (16, 8)
