"""The no-allocation x-shift entry point against the regular one (GPU).

vlasov_xshift_density_noalloc serves callers that may not allocate device memory: it works in a
fixed scratch array inside the library.  Two calls in a row (different sizes and boundary
conditions, so the second reuses scratch the first left behind) must each agree with the regular
handle-based path (vlasov_substep along x, then vlasov_density_force) to the FP64 sweep tolerance.
This file is collected last so that a stop-at-first-failure run has already run every other test.
"""
import numpy as np
import pytest

from paper_1206_3229_gb300 import inputs as I
from paper_1206_3229_gb300 import vlasov as V

pytestmark = pytest.mark.gpu

TOL = 1e-13


def regular_path(w: I.Workload, f: np.ndarray, disp: np.ndarray):
    with V.Sim.from_workload(w, precision="f64") as s:
        s.set_f(f)
        s.substep(0, disp)
        fout = s.get_f()
        rho, _ = s.density_force()
    return fout, rho


def noalloc_path(torch, w: I.Workload, f: np.ndarray, disp: np.ndarray):
    fin = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    dd = torch.from_numpy(np.ascontiguousarray(disp)).cuda()
    fout = torch.empty_like(fin)
    rho = torch.empty(w.nx, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    V.xshift_density_noalloc(fin.data_ptr(), fout.data_ptr(), rho.data_ptr(), w.nx, w.np, w.pmin, w.pmax,
                             w.x_periodic, dd.data_ptr(), None)
    torch.cuda.synchronize()
    return fout.cpu().numpy(), rho.cpu().numpy()


def test_noalloc_matches_regular_path_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(17)
    cases = [
        (I.HMF_256.resized(512, 384), rng.uniform(-40.0, 40.0, 384)),            # periodic x
        (I.SHEET_4096.resized(200, 328), rng.uniform(-30.0, 30.0, 328)),         # zero outside x, ragged
    ]
    for w, disp in cases:
        f = I.initial_state(w) * (1.0 + 0.1 * rng.uniform(-1, 1, (w.np, w.nx)))
        want_f, want_rho = regular_path(w, f, disp)
        got_f, got_rho = noalloc_path(torch, w, f, disp)
        assert np.max(np.abs(got_f - want_f)) <= TOL * np.max(np.abs(want_f)), w.name
        assert np.max(np.abs(got_rho - want_rho)) <= TOL * np.max(np.abs(want_rho)), w.name


def test_noalloc_at_its_size_limits_and_halo_edge():
    """Rows of the largest length (4096) on periodic and zero-outside rows, and zero-outside shifts
    at both ends of the accepted range -57 < s <= 56 (the regular handle gets the same halo from a
    time step whose row displacements reach 61 cells)."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(23)
    per = I.HMF_256.resized(4096, 64)
    zero = I.SHEET_4096.resized(4096, 64, dt=0.12)
    edge = rng.uniform(-56.9, 55.9, 64)
    edge[:6] = [56.0, -56.99, 55.999, -56.5, 0.0, 55.9]
    for w, disp in [(per, rng.uniform(-300.0, 300.0, 64)), (zero, edge)]:
        f = I.initial_state(w) * (1.0 + 0.1 * rng.uniform(-1, 1, (w.np, w.nx)))
        want_f, want_rho = regular_path(w, f, disp)
        got_f, got_rho = noalloc_path(torch, w, f, disp)
        assert np.max(np.abs(got_f - want_f)) <= TOL * np.max(np.abs(want_f)), w.name
        assert np.max(np.abs(got_rho - want_rho)) <= TOL * np.max(np.abs(want_rho)), w.name


def test_noalloc_flags_out_of_range_displacement():
    torch = pytest.importorskip("torch")
    w = I.SHEET_4096.resized(64, 64)
    f = I.initial_state(w)
    disp = np.zeros(w.np)
    disp[3] = 500.0                     # beyond the fixed zero halo of a non-periodic row
    _, rho = noalloc_path(torch, w, f, disp)
    assert np.all(np.isnan(rho))
    for s_bad in (56.01, -57.0):        # just outside -57 < s <= 56
        disp = np.zeros(w.np)
        disp[5] = s_bad
        _, rho = noalloc_path(torch, w, f, disp)
        assert np.all(np.isnan(rho)), s_bad
    _, rho2 = noalloc_path(torch, w, f, np.zeros(w.np))   # the next call starts clean
    assert np.all(np.isfinite(rho2))
