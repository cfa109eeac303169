"""Casimirs of Eq. (casimirs) on the GPU (vlasov_casimirs): the entropy, s(f) = -f log f, whose loss
the paper uses to measure information lost to the grid (Secs. 4.1-4.2), and the integral of f^2.
Compared with the FP64 oracle (pinned against closed forms in test_oracle_pins.py) evaluated on the
very values the handle stores (get_f), so that the check isolates the reduction itself."""
import numpy as np
import pytest

import oracle as O
from paper_1206_3229_gb300 import inputs as I
from paper_1206_3229_gb300 import vlasov as V

pytestmark = pytest.mark.gpu


def grid_of(w):
    return O.Grid(w.model, w.nx, w.np, w.xmin, w.xmax, w.pmin, w.pmax, w.x_periodic, w.p_periodic,
                  w.dt, w.eps, w.G)


@pytest.mark.parametrize("prec", ["f64", "fx64", "f64_native", "f32"])
def test_casimirs_match_the_oracle_on_the_stored_state(prec):
    w = I.HMF_256
    with V.Sim.from_workload(w, precision=prec) as s:
        s.set_f(I.initial_state(w))
        s.step(50)
        S, Q = s.casimirs()
        f = s.get_f()
    g = grid_of(w)
    assert S == pytest.approx(O.entropy(g, f), rel=1e-13)
    assert Q == pytest.approx(O.moments(g, f)["l2"], rel=1e-13)


def test_nodes_with_f_at_or_below_zero_add_nothing_to_the_entropy():
    w = I.HMF_256.resized(128, 96)
    f = I.initial_state(w)
    f[::5, ::3] = -0.01 * f.max()   # as spline undershoot leaves them
    f[1::7, ::4] = 0.0
    g = grid_of(w)
    with V.Sim.from_workload(w, precision="fx64") as s:
        s.set_f(f)
        S, Q = s.casimirs()
        fs = s.get_f()
    assert S == pytest.approx(O.entropy(g, fs), rel=1e-13)
    assert S == pytest.approx(O.entropy(g, np.where(fs > 0, fs, 0.0)), rel=1e-13)
    assert Q == pytest.approx(O.moments(g, fs)["l2"], rel=1e-13)


def test_casimirs_full_size_hmf_4096_initial_state():
    w = I.HMF_4096_UNSTABLE
    f0 = I.initial_state(w)
    with V.Sim.from_workload(w, precision="fx64") as s:
        s.set_f(f0)
        S, Q = s.casimirs()
        f = s.get_f()
    g = grid_of(w)
    assert S == pytest.approx(O.entropy(g, f), rel=1e-13)
    assert Q == pytest.approx(O.moments(g, f)["l2"], rel=1e-13)


def test_integer_free_streaming_conserves_every_casimir():
    """An integer-cell x-shift permutes the nodes: entropy and f^2 are unchanged (up to summation order)."""
    w = I.HMF_256.resized(128, 128)
    with V.Sim.from_workload(w, precision="f64") as s:
        s.set_f(I.initial_state(w))
        S0, Q0 = s.casimirs()
        s.substep(0, np.round(np.linspace(-20.0, 20.0, w.np)))
        S1, Q1 = s.casimirs()
    assert S1 == pytest.approx(S0, rel=1e-13) and Q1 == pytest.approx(Q0, rel=1e-13)


def test_casimirs_before_set_f_is_a_state_error():
    w = I.HMF_256.resized(64, 64)
    with V.Sim.from_workload(w, precision="fx64") as s:
        with pytest.raises(V.VlasovError) as e:
            s.casimirs()
        assert e.value.code == V.ESTATE
