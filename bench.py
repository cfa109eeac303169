#!/usr/bin/env python3
"""Benchmark of the Strang-split Vlasov step (arXiv:1206.3229, Sec. 3) on GB300.

Default workload: HMF model, 4096 x 4096 grid, theta in [-pi, pi) periodic, p in [-2, 2) with f = 0
outside, dt = 0.05, homogeneous waterbag (U = 0.55) with a 1e-6 cos(theta) mode, at FP64 accuracy.
A "step" is one full Strang step (x half-shift, force, p-shift, x half-shift, moments).

The headline storage mode is fx64: f held as 64-bit fixed point (round(f 2^(61-Ef)), 2^Ef four
times max|f|) and filtered with integer and FP32 units, accurate to about 2^-49 of 2^Ef per sweep:
the FP64 parity tolerance of the tests (1e-12 max f after 200 steps) holds for it as for IEEE
storage.  The IEEE-double storage (f64: same arithmetic, IEEE decode/encode), the hardware-FP64
filter (f64_native) and FP32 storage are timed beside it.

Prints ONE JSON line (rank 0).  value = cell-updates/s of the whole job (N ranks x Nx*Np*K / max
time).  Multi-GPU runs are independent replicas (no data-path collective); the NCCL process group
only provides the barrier and the max-over-ranks of the time.

--impl reference times the FP64 CPU oracle (the independent C implementation the tests use) on the
host cores, on the same workload and metric.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1206_3229_gb300 import inputs as I  # noqa: E402

METRIC = "Vlasov cell-updates/s"
UNIT = "cell-updates/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def workload_by_name(name: str) -> I.Workload:
    return I.WORKLOADS[name]


def oracle_grid(w):
    import oracle as O
    return O.Grid(w.model, w.nx, w.np, w.xmin, w.xmax, w.pmin, w.pmax, w.x_periodic, w.p_periodic, w.dt,
                  w.eps, w.G)


def cpu_oracle_timing(w: I.Workload, f0: np.ndarray, budget_s: float, max_steps: int) -> dict:
    """The FP64 oracle as it stands, on all host cores: whole Strang steps of the same workload."""
    import oracle as O
    cores = O.set_threads(os.cpu_count() or 1)
    g = oracle_grid(w)
    f = np.array(f0, copy=True)
    t0 = time.perf_counter()
    f, _ = O.run(g, f, 1, with_moments=True)
    t1 = time.perf_counter()
    per = t1 - t0
    more = int(max(0, min(max_steps - 1, budget_s / max(per, 1e-9) - 1)))
    if more:
        f, _ = O.run(g, f, more, with_moments=True)
    t2 = time.perf_counter()
    steps = 1 + more
    elapsed = t2 - t0
    # the paper compares with a serial code: the same oracle on one core, one step
    O.set_threads(1)
    s0 = time.perf_counter()
    O.run(g, f, 1, with_moments=True)
    single = time.perf_counter() - s0
    O.set_threads(cores)
    return {"value": w.cells * steps / elapsed, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{steps} full Strang step(s) of {w.name} ({w.nx}x{w.np}, FP64, moments each step) "
                      f"in {elapsed:.2f} s",
            "single_thread": {"value": w.cells / single, "unit": UNIT, "cores": 1,
                              "sample": f"1 full Strang step of {w.name} on one core in {single:.2f} s"}}


def sequential_single_grid(V, stream_handle, stream, mode: str = "fx64") -> dict:
    """The requests of a serving stream one at a time on the single-grid path `mode` (measured, not
    estimated): each request is created, given its initial state on the device, run for its step
    count and read back.  Device time: CUDA events around each request's steps (its first step,
    which captures the step graphs, is timed too); wall time: everything, creation included.  The
    last moment record of each request is the accuracy reference of the batched forms."""
    import torch
    st_ = torch.cuda.ExternalStream(stream_handle)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dev_ms = 0.0
    last = []
    t0 = time.perf_counter()
    for (w, steps, _t) in stream:
        with V.Sim.from_workload(w, precision=mode, stream=stream_handle) as s:
            s.init_workload(w)
            e0.record(st_)
            s.step(steps)
            e1.record(st_)
            e1.synchronize()
            dev_ms += e0.elapsed_time(e1)
            last.append(s.moments()[-1])
    return {"mode": mode, "device_s": dev_ms * 1e-3, "wall_s": time.perf_counter() - t0, "last": np.array(last)}


def accuracy_vs(res, seq_last, stream) -> dict:
    """|dM| = | |M| of the batched result - |M| of the one-at-a-time FP64-accurate run | for every
    completed request (the magnetisation modulus; for the sheet the same cos/sin moments of x)."""
    dM = []
    for q, (r, (w, st, _t)) in enumerate(zip(res, stream)):
        if r.status != 0:
            continue
        mb = math.hypot(r.last.Mx, r.last.My)
        ms = math.hypot(seq_last[q, 2], seq_last[q, 3])
        dM.append((abs(mb - ms), w.model, w.nx, st))
    v = np.array([d[0] for d in dM]) if dM else np.zeros(0)
    worst = sorted(dM, reverse=True)[:5]
    by_model = {}
    for m in ("hmf", "ring", "sheet"):
        vm = np.array([d[0] for d in dM if d[1] == m])
        if len(vm):
            by_model[m] = {"n": int(len(vm)), "max": float(vm.max()), "frac_within_1e-5": float(np.mean(vm <= 1e-5))}
    return {"dM_all_max": float(v.max()) if len(v) else None, "dM_by_model": by_model,
            "dM_p99": float(np.percentile(v, 99)) if len(v) else None,
            "dM_median": float(np.median(v)) if len(v) else None,
            "frac_within_1e-5": float(np.mean(v <= 1e-5)) if len(v) else None,
            "n_compared": int(len(v)),
            "worst": [{"dM": d[0], "model": d[1], "n": d[2], "steps": d[3]} for d in worst]}


def serving_benchmark(V, stream_handle, slots: int, budget_bytes: int, precision: str, stream, rate: float) -> dict:
    """The seeded 512-request serving stream in the batched form with `precision` storage, by
    continuous batching at the given arrival rate.  Reports aggregate cell-updates/s over the
    makespan and p50/p99 time-to-result (completion of the last step on the GPU minus arrival)."""
    sizes = (256, 512, 1024, 2048)
    # launch shape of the batched sweeps: the project's autotuner, run once before anything is timed
    # (later batches of this max_n and precision use the shape it picked)
    shape, shape_ms = V.batch_autotune(max(sizes), precision, stream_handle)
    reqs = [V.request_from_workload(w, st, t) for (w, st, t) in stream]
    res, makespan = V.serve(reqs, slots, budget_bytes, max_n=max(sizes), stream=stream_handle, precision=precision)
    ok = [r.status == 0 for r in res]
    work = sum(w.cells * st for (w, st, _t), good in zip(stream, ok) if good)
    lat = np.array([r.done_s - r.arrival_s for r, good in zip(res, ok) if good])
    return {"requests": len(reqs), "completed": int(sum(ok)), "slots": slots, "mem_budget_gb": budget_bytes / 2 ** 30,
            "precision": precision,
            "launch_shape": {"rows_per_cta": shape[0], "tiles_per_cta": shape[1],
                             "autotune_ms_per_batched_step": {f"{r}x{t}": round(v, 4) for (r, t), v in shape_ms.items()}},
            "dtype": {"f32": "f32 storage, FP64-accurate displacements (exact fixed-point ring force) and moment sums",
                      "fx64": "int64 fixed point + f32 (FP64-accurate), as the single-grid fx64 path"}[precision],
            "aggregate_value": work / makespan, "unit": UNIT, "makespan_s": makespan, "arrival_rate_per_s": rate,
            "latency_p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
            "latency_p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
            "_results": res, "_work": work}


def serving_section(V, stream_handle, slots: int, budget_bytes: int) -> dict:
    """Both batched forms on the same stream, the same requests measured one at a time on the
    single-grid FX64 path, and every request's |dM| against that run.  Offered load: 80% of the FP32
    batched capacity measured on a calibration burst in the same run."""
    sizes = (256, 512, 1024, 2048)
    cal = I.serving_stream(48, seed=55, sizes=sizes, step_scale=0.1, rate_per_s=1e9)
    creqs = [V.request_from_workload(w, st, 0.0) for (w, st, _t) in cal]
    V.batch_autotune(max(sizes), "f32", stream_handle)
    _, mk = V.serve(creqs, slots, budget_bytes, max_n=max(sizes), stream=stream_handle, precision="f32")
    capacity = sum(w.cells * st for (w, st, _t) in cal) / mk
    rate = 0.8 * capacity / (float(np.mean([n * n for n in sizes])) * 1050.0)
    stream = I.serving_stream(512, seed=5, sizes=sizes, rate_per_s=rate)
    out = {"requests": len(stream), "capacity_calibration": capacity, "offered_load_of_capacity": 0.8}
    seq = sequential_single_grid(V, stream_handle, stream, "fx64")
    seq_work = sum(w.cells * st for (w, st, _t) in stream)
    out["sequential_fx64"] = {"device_s": seq["device_s"], "wall_s": seq["wall_s"],
                              "value_device": seq_work / seq["device_s"], "unit": UNIT,
                              "note": "the 512 requests run one at a time on the single-grid FX64 path (measured)"}
    for prec in ("f32", "fx64"):
        r = serving_benchmark(V, stream_handle, slots, budget_bytes, prec, stream, rate)
        res, work = r.pop("_results"), r.pop("_work")
        r.update(accuracy_vs(res, seq["last"], stream))
        r["speedup_vs_sequential_fx64_device"] = seq["device_s"] / r["makespan_s"] * (work / seq_work)
        r["speedup_vs_sequential_fx64_wall"] = seq["wall_s"] / r["makespan_s"] * (work / seq_work)
        out[prec] = r
    ok = [p for p in ("f32", "fx64") if out[p]["dM_all_max"] is not None and out[p]["dM_all_max"] <= 1e-5
          and out[p]["completed"] == out[p]["requests"]]
    out["headline_form"] = max(ok, key=lambda p: out[p]["aggregate_value"]) if ok else None
    out["headline_rule"] = ("the fastest batched form whose every result is within |dM| <= 1e-5 of the "
                            "one-at-a-time FP64-accurate run")
    return out


DTYPE = {"fx64": "int64 fixed point + f32 (FP64-accurate)", "f64": "f64 storage, int64 + f32 arithmetic (FP64-accurate)",
         "f64_native": "f64", "f32": "f32", "bf16": "bf16 storage, f32 arithmetic (experiment)"}
# Source files whose kernels each storage mode's sweeps run (for matching stored ncu traffic).
KERNEL_SOURCES = {"fx64": ("shift_fx.cu",), "f64": ("shift_f64e.cu",), "f64_native": ("shift_kernels.cu",),
                  "f32": ("shift_kernels.cu",), "bf16": ("shift_kernels.cu",)}
COMMON_SOURCES = ("emul.cuh", "ptx.cuh", "shift_common.cuh", "vlasov_internal.cuh", "fixed_point.cuh")


def kernel_source_hash(precision: str) -> str:
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[precision] + COMMON_SOURCES:
        with open(os.path.join(ROOT, "paper_1206_3229_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def stored_traffic(precision: str, slot: str):
    """DRAM bytes per launch of a sweep kernel from the committed ncu summary, or None when the
    kernel sources changed since that capture (the summary records the source hash)."""
    try:
        with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as fh:
            d = json.load(fh)
        e = d[precision]
        if e["source_hash"] != kernel_source_hash(precision):
            return None
        return e["bytes_per_launch"].get(slot)
    except Exception:
        return None


def reduce_max(x: float, world: int, device: str) -> float:
    """Max of a per-rank number over the process group (identity for one rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, cells: int, steps: int, seconds_max: float) -> float:
    """Whole-job cell-updates/s: every rank advances its own grid `steps` times (weak scaling)."""
    return world * cells * steps / seconds_max


def bench_config(w: I.Workload, gpus: int, accuracy: str) -> dict:
    """The `config` object of both arms' JSON lines (same keys and values for the same run)."""
    cells = w.nx * w.np
    return {"workload": w.name, "grid": f"{w.nx}x{w.np}", "dt": w.dt, "accuracy": accuracy,
            "parallelism": "replicas" if gpus > 1 else "single",
            "l2": f"inputs larger than L2: each sweep streams {16 * cells / 1e6:.0f} MB at FP64 (read + write) "
                  "against a 129 MB L2"}


ACCURACY = {"fx64": "fp64", "f64": "fp64", "f64_native": "fp64", "f32": "fp32", "bf16": "bf16"}


def config_checks(V, stream_handle) -> dict:
    """The three large workloads at their own sizes and step counts, in FX64 (FP64-accurate) and FP32
    storage, each from its waterbag generated on the device: the growth rate of |M| of the unstable
    HMF waterbag against the waterbag dispersion relation (gamma = sqrt(1/2 - p0^2), p0^2 = 3 <p^2> of
    the discrete f0), |dM(t)| of FP32 against FX64, and mass and energy drift (mass leaves through the
    zero-outside edges once the distribution reaches them)."""
    out = {}
    for w in (I.HMF_4096_UNSTABLE, I.RING_2048, I.SHEET_4096):
        hist, secs = {}, {}
        for prec in ("fx64", "f32"):
            with V.Sim.from_workload(w, precision=prec, stream=stream_handle) as s:
                s.init_workload(w)
                t0 = time.perf_counter()
                parts, left = [], w.steps
                while left:
                    k = min(left, 4000)
                    s.step(k)
                    parts.append(s.moments())
                    left -= k
                secs[prec] = time.perf_counter() - t0
                hist[prec] = np.concatenate(parts)
        a, b = hist["fx64"], hist["f32"]
        Ma, Mb = np.hypot(a[:, 2], a[:, 3]), np.hypot(b[:, 2], b[:, 3])
        d = np.abs(Ma - Mb)
        over = np.nonzero(d > 1e-5)[0]
        mass_def = np.abs(a[:, 1] - a[0, 1])
        leak = np.nonzero(mass_def > 1e-12)[0]
        e = {"steps": w.steps, "grid": f"{w.nx}x{w.np}", "wall_s": secs,
             "dM_vs_fp64_max": float(d.max()),
             "dM_vs_fp64_first_over_1e-5": ({"step": int(over[0]) + 1, "t": float(a[over[0], 0]),
                                             "M_fp64": float(Ma[over[0]])} if len(over) else None),
             "mass_drift_max": float(mass_def.max()),
             "mass_conserved_until_t": float(a[leak[0], 0]) if len(leak) else float(a[-1, 0]),
             "energy_rel_drift_end": float((a[-1, 6] - a[0, 6]) / abs(a[0, 6]))}
        if len(leak):
            k = max(int(leak[0]) - 1, 0)
            e["energy_rel_drift_before_outflow"] = float((a[k, 6] - a[0, 6]) / abs(a[0, 6]))
        if w.model == "hmf":
            f0 = I.initial_state(w)
            pj = w.pmin + np.arange(w.np) * w.dp
            gth = math.sqrt(0.5 - 3 * float(np.sum(f0 * (pj ** 2)[:, None])) * w.dx * w.dp)
            for prec, h in (("fx64", a), ("f32", b)):
                M = np.hypot(h[:, 2], h[:, 3])
                sel = (M > 1e-5) & (M < 1e-3)
                g = float(np.polyfit(h[sel, 0], np.log(M[sel]), 1)[0])
                e[f"growth_rate_{prec}"] = g
                e[f"growth_rate_rel_err_{prec}"] = (g - gth) / gth
            e["growth_rate_theory"] = gth
        out[w.name] = e
    return out


def ring_section(V, stream_handle) -> dict:
    """The ring workload (2048^2): microseconds per force launch of each circulant-convolution method
    (vlasov_ring_timings) and ms per whole step with each method, in FX64 and FP32 storage."""
    import torch
    st_ = torch.cuda.ExternalStream(stream_handle)
    w = I.RING_2048
    out = {}
    for prec in ("fx64", "f32"):
        with V.Sim.from_workload(w, precision=prec, stream=stream_handle) as s:
            s.init_workload(w)
            s.step(5)
            s.sync()
            default = s.ring_method
            r = {"default_method": default, "force_us": s.ring_timings(200), "ms_per_step": {}}
            for m in ("fixed", "direct", "fft", "fft_f32"):
                s.ring_method = m
                s.step(8)
                s.sync()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st_)
                s.step(64)
                e1.record(st_)
                e1.synchronize()
                r["ms_per_step"][m] = e0.elapsed_time(e1) / 64
            s.ring_method = default
        out[prec] = r
    return out


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    f0 = I.initial_state(w)
    import oracle as O
    cores = O.set_threads(os.cpu_count() or 1)
    g = oracle_grid(w)
    f = np.array(f0, copy=True)
    # warm-up and sizing: each "step" is one full oracle Strang step of the workload
    t0 = time.perf_counter()
    f, _ = O.run(g, f, max(args.warmup, 1), with_moments=True)
    per = (time.perf_counter() - t0) / max(args.warmup, 1)
    steps = int(max(1, min(args.steps, 150.0 / max(per, 1e-9))))
    t0 = time.perf_counter()
    f, _ = O.run(g, f, steps, with_moments=True)
    el = time.perf_counter() - t0
    v = w.cells * steps / el
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(w, args.gpus, "fp64"), "precision": "f64 (the FP64 oracle)",
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{steps} full Strang steps of {w.name} on {cores} host threads"
                                       + ("" if steps == args.steps else f" (capped from {args.steps})")},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=I.HMF_4096_UNSTABLE.name, choices=sorted(I.WORKLOADS))
    ap.add_argument("--precision", default="fx64", choices=["f64", "fx64", "f32", "f64_native", "bf16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-f32", action="store_true", help="skip the secondary measurements of the other storage modes")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-serve", action="store_true", help="skip the batched serving-stream measurement")
    ap.add_argument("--no-checks", action="store_true",
                    help="skip the full-length workload checks and the ring-method timings")
    ap.add_argument("--serve-slots", type=int, default=64)
    ap.add_argument("--serve-budget-gb", type=float, default=8.0)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    w = workload_by_name(args.workload)
    if args.impl == "reference":
        return run_reference(args, w)

    import torch
    import torch.distributed as dist
    from paper_1206_3229_gb300 import vlasov as V

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    f0 = I.initial_state(w)
    cells = w.cells
    esz = {"f32": 4, "bf16": 2}.get(args.precision, 8)
    stream = torch.cuda.Stream()
    sim = V.Sim.from_workload(w, precision=args.precision, stream=stream.cuda_stream)
    sim.set_f(f0)

    # warm-up (the first step captures the CUDA graphs)
    sim.step(args.warmup)
    sim.sync()
    sim.moments()

    # ---- timed region: K graph-launched steps, device events on the solver's stream
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0.record(stream)
        sim.step(args.steps)
        e1.record(stream)
        e1.synchronize()
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    ms_max = reduce_max(ms, world, "cuda")
    hist = sim.moments()
    value = job_value(world, cells, args.steps, ms_max * 1e-3)

    # ---- per-kernel durations (eager launches with events on the same stream)
    slot_ms = sim.step_timed(4)
    names = sim.slot_names()
    peak_gbs, peak_src = _peaks()
    shift_bytes = 2.0 * cells * esz   # one read + one write of f per sweep launch (the bytes it moves)
    dom = int(np.argmax(slot_ms))
    dom_name = names[dom]
    # the per-sweep traffic model (one read + one write of f per sweep and output) counts the fused
    # launch, which does the arithmetic of two sweeps on one read and one write, as two sweeps
    sweeps_in = 2 if dom_name == "xshift_fused" else 1
    model_bytes = sweeps_in * shift_bytes
    t_dom = slot_ms[dom] * 1e-3
    achieved = model_bytes / t_dom / 1e9 if "shift" in dom_name else None
    achieved_phys = shift_bytes / t_dom / 1e9 if "shift" in dom_name else None
    # HBM round trips of f per step: 3 sweeps, or 2 when the second x half-shift of a step and the
    # first of the next run as one launch (the row stays on chip between them)
    sweeps = 2 if sim.fused_x and args.steps >= 2 else 3
    step_gbs = sweeps * shift_bytes / (ms_max / args.steps * 1e-3) / 1e9
    traffic = stored_traffic(args.precision, dom_name)
    roofline = {"bound": "hbm", "kernel": dom_name, "achieved": achieved, "peak": peak_gbs, "unit": "GB/s",
                "frac": (achieved / peak_gbs) if achieved else None,
                "frac_model": (achieved / peak_gbs) if achieved else None,
                "frac_physical": (achieved_phys / peak_gbs) if achieved_phys else None,
                "achieved_physical": achieved_phys, "sweeps_in_launch": sweeps_in,
                "traffic": traffic, "algorithmic_bytes": model_bytes, "physical_bytes": shift_bytes,
                "launch_ms": float(slot_ms[dom]), "peak_source": peak_src,
                "note": ("achieved/frac: the per-sweep model, 2 x sizeof(f) per output and sweep, for the two sweeps "
                         "of arithmetic the fused launch does; frac_physical: the one read and one write of f it "
                         "makes (traffic: its ncu DRAM bytes).  Bound by instruction issue, not HBM (profiles/)")
                if dom_name == "xshift_fused" else None,
                "per_kernel_ms": {n: round(float(v), 5) for n, v in zip(names, slot_ms)},
                "per_kernel_gbs": {n: round(shift_bytes / (v * 1e-3) / 1e9, 1) for n, v in zip(names, slot_ms)
                                   if "shift" in n and not n.endswith("filters")}}

    # ---- Casimirs of the state after the timed steps (entropy and integral of f^2): one synced call
    cas_ms = []
    for _ in range(3):
        c0 = time.perf_counter()
        S_ent, Q_l2 = sim.casimirs()
        cas_ms.append((time.perf_counter() - c0) * 1e3)
    casimirs = {"entropy": S_ent, "l2": Q_l2, "ms_per_call": min(cas_ms),
                "read_gbs": cells * esz / (min(cas_ms) * 1e-3) / 1e9,
                "note": "vlasov_casimirs: one FP64 log per cell (bound by the FP64 pipe, not HBM), host-timed "
                        "call including its launch and synchronisation"}

    # ---- end to end through the public API with host buffers
    pinned = torch.empty((w.np, w.nx), dtype=torch.float64, pin_memory=True).numpy()
    pinned[...] = f0
    out = torch.empty((w.np, w.nx), dtype=torch.float64, pin_memory=True).numpy()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.set_f(pinned)
    sim.step(args.steps)
    m = sim.moments()
    sim.get_f(out)
    t1 = time.perf_counter()
    e2e_s = reduce_max(t1 - t0, world, "cuda")
    e2e = {"value": job_value(world, cells, args.steps, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": cells * 8 / args.steps,
           "d2h_bytes_per_step": (cells * 8 + 64 * args.steps) / args.steps,
           "note": "one job per timed region: vlasov_set_f from pinned host f0, K steps, moments and f back"}
    launches = sim.launches(args.steps)

    # ---- secondary: the other storage modes on the same workload (same timing rules)
    others = {}
    if not args.no_f32:
        for prec in [p for p in ("fx64", "f64", "f64_native", "f32", "bf16") if p != args.precision]:
            s2 = V.Sim.from_workload(w, precision=prec, stream=stream.cuda_stream)
            s2.set_f(f0)
            s2.step(args.warmup)
            s2.sync()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            s2.step(args.steps)
            a1.record(stream)
            a1.synchronize()
            ms2 = a0.elapsed_time(a1)
            sl2 = s2.step_timed(4)
            eb = {"f32": 4, "bf16": 2}.get(prec, 8)
            sw2 = 2 if s2.fused_x and args.steps >= 2 else 3
            others[prec] = {"value": world * cells * args.steps / (ms2 * 1e-3), "ms_per_step": ms2 / args.steps,
                            "hbm_sweeps_per_step": sw2,
                            "hbm_roofline_frac_step": sw2 * 2.0 * cells * eb / (ms2 / args.steps * 1e-3) / 1e9 / peak_gbs,
                            "per_kernel_ms": {n: round(float(v), 5) for n, v in zip(s2.slot_names(), sl2)}}
            s2.close()

    # ---- secondary: the global-spline variant (Eq. tridiagsys, Tables 1-2) on the same workload.
    # Its sweeps run a 64-tap filter per output in IEEE arithmetic: bound by the FP64 pipe (FP64) or
    # by shared-memory reads (FP32); the roofline below is the x-shift's multiply-add rate against
    # the nominal FP64 rate (2 DFMA/clock/SM) or FP32 rate (128 FFMA/clock/SM) at 152 SMs, 2070 MHz.
    gspline = {}
    if not args.no_f32:
        for prec, peak_tfma in (("f64_native", 152 * 2 * 2.07e9 / 1e12), ("f32", 152 * 128 * 2.07e9 / 1e12)):
            s2 = V.Sim.from_workload(w, precision=prec, stream=stream.cuda_stream)
            s2.spline = "gs"
            s2.set_f(f0)
            s2.step(2)
            s2.sync()
            k2 = min(args.steps, 10)
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            s2.step(k2)
            a1.record(stream)
            a1.synchronize()
            ms2 = a0.elapsed_time(a1) / k2
            sl2 = dict(zip(s2.slot_names(), s2.step_timed(2)))
            tx = float(sl2["xshift_step1"])
            ach = cells * 64 / (tx * 1e-3) / 1e12
            gspline[prec] = {"value": world * cells / (ms2 * 1e-3), "ms_per_step": ms2,
                             "per_kernel_ms": {n: round(float(v), 5) for n, v in sl2.items()},
                             "roofline": {"bound": "alu", "kernel": "gs_xshift", "achieved": ach, "peak": peak_tfma,
                                          "unit": "TFMA/s", "frac": ach / peak_tfma,
                                          "peak_source": "nominal unit count x max SM clock"}}
            s2.close()

    checks = config_checks(V, stream.cuda_stream) if (rank == 0 and not args.no_checks) else None
    rings = ring_section(V, stream.cuda_stream) if (rank == 0 and not args.no_checks) else None

    serving = None
    if not args.no_serve and rank == 0:
        serving = serving_section(V, stream.cuda_stream, args.serve_slots, int(args.serve_budget_gb * 2 ** 30))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_timing(w, f0, args.cpu_budget, 50)

    sim.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
                "config": bench_config(w, world, ACCURACY[args.precision]), "precision": args.precision,
                "hbm_roofline_frac_step": step_gbs / peak_gbs,
                "hbm_sweeps_per_step": sweeps,
                "hbm_frac_step_at_3_sweeps": 3 * shift_bytes / (ms_max / args.steps * 1e-3) / 1e9 / peak_gbs,
                "roofline": roofline,
                "cpu_baseline": cpu,
                "e2e": e2e,
                "gpu_launches": launches,
                "clocks": clk.summary(),
                "moments_last": {"t": float(hist[-1, 0]), "mass": float(hist[-1, 1]),
                                 "M": float(np.hypot(hist[-1, 2], hist[-1, 3])), "energy": float(hist[-1, 6])}
                if len(hist) else None,
                "other_precisions": others,
                "global_spline": gspline,
                "casimirs": casimirs,
                "config_checks": checks,
                "ring": rings,
                "serving": serving}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
