"""The three large workloads at their own sizes and step counts, on the GPU, against the FP64 oracle's
full-length runs (tests/golden/config_*.npz, written by tests/golden/make_config_references.py,
which calls only the oracle).

* After 200 steps the FP64-accurate path (FX64 storage) agrees with the oracle on its strided
  sub-grid of f within what its arithmetic allows: each sweep rounds the FP32 residual sum of the
  filter to at most 2^-47 of the fixed-point bound 2^Ef (four to eight times max f), so 3 x 200
  sweeps add up to at most 600 * 2^-47 * 2^Ef even when every rounding falls the same way (3.4e-11 of
  max f for the sheet, 2.7e-11 for the ring, 2.9e-11 for the HMF waterbag).  Measured: 1.3e-11
  (sheet: at two mirror points of the collapsed core where the same rounding recurs every step),
  2.7e-12 (ring), 3.2e-13 (HMF).  The moments after 200 steps agree to 1e-12.
* Over the whole run the moment histories agree.  The unstable HMF waterbag amplifies every
  difference in its seed mode at the rate it amplifies the mode itself, so |dM(t)| is held relative
  to |M(t)| (measured: 5.3e-10 of |M| at most); the ring and the sheet are held absolutely.
* The growth rate of |M| of the unstable waterbag (linearised Eqs. vlasoveq, hmfmeanforce, mxmydef;
  dispersion relation of the waterbag) is within 3% of sqrt(1/2 - p0^2), p0^2 = 3 <p^2> of the
  discrete f0, at the full 4096^2 and 1000 steps, in FX64 and in FP32 storage.
* FP32 storage: |dM(t)| <= 1e-5 against the oracle is asserted over the stretch where it holds; the
  step where it first fails is recorded in the design notes, not hidden by a looser bound.
"""
import math
import os

import numpy as np
import pytest

from paper_1206_3229_gb300 import inputs as I
from paper_1206_3229_gb300 import vlasov as V

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def reference(w):
    path = os.path.join(GOLDEN, f"config_{w.name}.npz")
    if not os.path.exists(path):
        pytest.skip(f"no oracle reference for {w.name}")
    return np.load(path)


def run(w, prec, snap=200):
    """Full-length run from the device-generated waterbag: moments of every step, f at `snap` and at the end."""
    with V.Sim.from_workload(w, precision=prec) as s:
        s.init_workload(w)
        s.step(snap)
        m1, f1 = s.moments(), s.get_f()
        s.step(w.steps - snap)
        m2, f2 = s.moments(), s.get_f()
    return np.concatenate([m1, m2]), f1, f2


def modulus(m):
    return np.hypot(m[:, 2], m[:, 3])


# absolute bounds on the moment histories over the whole run (FX64 vs oracle)
ABS = {"ring_2048": 1e-11, "sheet_4096": 1e-11}


@pytest.mark.parametrize("w", [I.HMF_4096_UNSTABLE, I.RING_2048, I.SHEET_4096], ids=lambda w: w.name)
def test_full_size_run_matches_oracle_fp64(w):
    ref = reference(w)
    sx, sp = (int(v) for v in ref["stride"])
    m, f200, fend = run(w, "fx64")
    mo = ref["moments"]
    assert m.shape == mo.shape
    assert np.max(np.abs(m[:, 0] - mo[:, 0])) <= 1e-9
    fmax = float(I.initial_state(w).max())
    Ef = math.frexp(fmax)[1] + 2                      # the library's bound: 2^Ef >= 4 max f
    bound = 3 * 200 * 2.0 ** -47 * 2.0 ** Ef / fmax
    e_fx = float(np.max(np.abs(f200[::sx, ::sp] - ref["f200"]))) / fmax
    assert e_fx <= bound, (e_fx, bound)
    assert np.max(np.abs(m[:200, 1:7] - mo[:200, 1:7])) <= 1e-12
    Mg, Mo = modulus(m), modulus(mo)
    if w.model == "hmf":
        assert np.max(np.abs(Mg - Mo) / np.maximum(Mo, 1e-300)) <= 2e-9
        assert np.max(np.abs(m[:, [1, 6]] - mo[:, [1, 6]])) <= 1e-12
    else:
        assert np.max(np.abs(Mg - Mo)) <= ABS[w.name]
        assert np.max(np.abs(m[:, 1:7] - mo[:, 1:7])) <= ABS[w.name]
    # the end state, sampled.  After saturation the unstable waterbag filaments down to the grid
    # scale, so the 5e-10 relative agreement of M becomes 2.2e-7 max f (measured) at the sharpest
    # gradients of f after 1000 steps; the ring and the sheet stay far closer.
    assert np.max(np.abs(fend[::sx, ::sp] - ref["fend"])) <= (1e-6 if w.model == "hmf" else 1e-10) * fmax


@pytest.mark.parametrize("prec", ["fx64", "f32"])
def test_unstable_waterbag_growth_rate_at_full_size(prec):
    w = I.HMF_4096_UNSTABLE
    f0 = I.initial_state(w)
    pj = w.pmin + np.arange(w.np) * w.dp
    gamma_th = math.sqrt(0.5 - 3 * float(np.sum(f0 * (pj ** 2)[:, None])) * w.dx * w.dp)
    with V.Sim.from_workload(w, precision=prec) as s:
        s.init_workload(w)
        s.step(w.steps)
        m = s.moments()
    M = modulus(m)
    sel = (M > 1e-5) & (M < 1e-3)
    assert sel.sum() > 100
    gamma = np.polyfit(m[sel, 0], np.log(M[sel]), 1)[0]
    assert abs(gamma - gamma_th) <= 0.03 * gamma_th, (gamma, gamma_th)


def test_fp32_magnetisation_against_oracle_where_the_bound_holds():
    """FP32 storage cannot hold the unstable waterbag's 1e-6 seed mode exactly (FP32 resolves 6e-8 of
    f): the growing mode comes out about 3% off (measured 3.1% at step 100, 2.9% at step 200), and
    the instability keeps that fraction while |M| grows.  So the FP32 bound |dM| <= 1e-5 holds while
    |M| stays below 1e-5 / 3% = 3e-4 and fails after (first at step 297, |M| = 3.5e-4); the ring holds
    it for its first 600 steps (first fails at step 614).  Asserted where it holds; the failing
    steps are reported with the bench line, not hidden by a looser bound."""
    w = I.HMF_4096_UNSTABLE
    ref = reference(w)
    m, _, _ = run(w, "f32")
    Mo, Mg = modulus(ref["moments"]), modulus(m)
    lin = (Mo > 1e-6) & (Mo < 1e-3)
    assert np.max(np.abs(Mg[lin] - Mo[lin]) / Mo[lin]) <= 0.05
    k = int(np.nonzero(Mo > 3e-4)[0][0])
    assert np.max(np.abs(Mg[:k] - Mo[:k])) <= 1e-5
    assert np.max(np.abs(m[:, 1] - ref["moments"][:, 1])) <= 1e-5   # mass
    w = I.RING_2048
    ref = reference(w)
    m, _, _ = run(w, "f32")
    Mo, Mg = modulus(ref["moments"]), modulus(m)
    assert np.max(np.abs(Mg[:600] - Mo[:600])) <= 1e-5
    assert np.max(np.abs(m[:, 1] - ref["moments"][:, 1])) <= 1e-5
