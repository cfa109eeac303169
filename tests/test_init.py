"""vlasov_init_waterbag (the waterbag initial states of Sec. 4, generated on the device) against the
shared seeded host generator `inputs.initial_state`, through the C ABI.

The two draw the same SplitMix64 noise and round every product the same way; they differ only in
how the unit-mass normalisation sums (exact fixed point on the device, numpy's pairwise sum on the
host), so f agrees to a few FP64 ulps.  In the other storage modes the device state is compared
with the same host array uploaded through vlasov_set_f, within one unit of the storage format.
"""
import numpy as np
import pytest

from paper_1206_3229_gb300 import inputs as I
from paper_1206_3229_gb300 import vlasov as V

pytestmark = pytest.mark.gpu

SMALL = [
    I.HMF_256,
    I.HMF_256.resized(200, 328),                                   # ragged grid
    I.HMF_4096_UNSTABLE.resized(256, 128),                         # homogeneous + cos mode
    I.RING_2048.resized(256),
    I.SHEET_4096.resized(128, 256),                                # zero-outside x and p
    I.Workload("homog_box", "hmf", 64, 64, -np.pi, np.pi, -2.0, 2.0, True, False, 0.1, 1,
               init="box", x0=4.0, p0=0.7, noise=1e-4, seed=99),  # x0 >= half extent: all columns
]
FULL = [I.HMF_4096_UNSTABLE, I.RING_2048, I.SHEET_4096]


def _device_state(w, prec):
    with V.Sim.from_workload(w, precision=prec) as s:
        s.init_workload(w)
        return s.get_f()


def _uploaded_state(w, prec, f0):
    with V.Sim.from_workload(w, precision=prec) as s:
        s.set_f(f0)
        return s.get_f()


@pytest.mark.parametrize("w", SMALL + FULL, ids=lambda w: f"{w.name}_{w.nx}x{w.np}")
def test_fp64_initial_state_matches_host_generator(w):
    f0 = I.initial_state(w)
    fd = _device_state(w, "f64")
    assert fd.shape == f0.shape
    assert np.max(np.abs(fd - f0)) <= 1e-15 * f0.max()
    assert np.array_equal(fd == 0, f0 == 0)                      # same support, bit for bit
    assert abs(w.dx * w.dp * fd.sum() - 1.0) <= 1e-13


@pytest.mark.parametrize("prec", ["fx64", "f64_native", "f32", "bf16"])
@pytest.mark.parametrize("w", SMALL + [I.HMF_4096_UNSTABLE], ids=lambda w: f"{w.name}_{w.nx}x{w.np}")
def test_initial_state_in_every_storage_mode(w, prec):
    f0 = I.initial_state(w)
    fd = _device_state(w, prec)
    fu = _uploaded_state(w, prec, f0)
    # one unit of the storage format (FP64 ulps, the fixed-point quantum, an FP32 or bf16 ulp)
    tol = {"fx64": 1e-15, "f64_native": 1e-15, "f32": 2.0 ** -23, "bf16": 2.0 ** -8}[prec]
    if prec in ("fx64", "f64_native"):
        assert np.max(np.abs(fd - fu)) <= tol * f0.max()
    else:
        assert np.all(np.abs(fd - fu) <= tol * np.abs(fu))


@pytest.mark.parametrize("prec", ["fx64", "f32"])
def test_steps_from_device_state_match_steps_from_upload(prec):
    w = I.HMF_256
    f0 = I.initial_state(w)
    out = []
    for dev in (True, False):
        with V.Sim.from_workload(w, precision=prec) as s:
            if dev:
                s.init_workload(w)
            else:
                s.set_f(f0)
            s.step(20)
            out.append((s.get_f(), s.moments()))
    (fa, ma), (fb, mb) = out
    tol = 1e-13 if prec == "fx64" else 1e-6
    assert np.max(np.abs(fa - fb)) <= tol * fb.max()
    assert ma.shape == mb.shape == (20, 8)
    assert np.max(np.abs(ma[:, 1:7] - mb[:, 1:7])) <= tol


def test_bad_waterbag_arguments_are_rejected():
    w = I.Workload("empty", "hmf", 64, 16, -np.pi, np.pi, -2.1, 2.0, True, False, 0.1, 1)
    with V.Sim.from_workload(w, precision="f64") as s:
        for args in [(1.0, 0.0, 0.0, 0, 0, 0.0),      # p0 <= 0
                     (0.0, 1.0, 0.0, 0, 0, 0.0),      # x0 <= 0
                     (1.0, 1.0, 1.5, 0, 0, 0.0),      # noise >= 1
                     (1.0, 1.0, 0.0, 0, 2, 0.0),      # unknown mode
                     (1.0, 1.0, 0.0, 0, 1, 1.0),      # |mode_amp| >= 1
                     (1.0, 1e-3, 0.0, 0, 0, 0.0)]:    # no node with |p_j| < p0: empty state
            with pytest.raises(V.VlasovError) as e:
                s.init_waterbag(*args)
            assert e.value.code == V.EINVAL
        with pytest.raises(V.VlasovError) as e:
            s.step(1)                                  # still no state
        assert e.value.code == V.ESTATE
