"""Failure detection without a GPU fault: a bounded device wait that expires.

Every staged sweep waits for its rows with a %globaltimer-bounded mbarrier wait and, when the wait
gives up, records a timeout code in the handle's device error flag and returns.  vlasov_test_expire_wait
drives that path on purpose -- one CTA waits, with a short limit, on a barrier that nothing arrives
on and no copy completes -- so no copy is in flight and the context stays usable.  The host must then
see VLASOV_ETIMEOUT at the next syncing call, and the handle (and a fresh one) must run clean after.
"""
import numpy as np
import pytest

from paper_1206_3229_gb300 import inputs as I
from paper_1206_3229_gb300 import vlasov as V

pytestmark = pytest.mark.gpu


def test_expired_wait_is_reported_and_the_handle_recovers():
    w = I.HMF_256.resized(128)
    f0 = I.initial_state(w)
    with V.Sim.from_workload(w, precision="fx64") as s:
        s.set_f(f0)
        s.step(3)
        s.sync()
        s.test_expire_wait(1_000_000)                 # 1 ms limit
        with pytest.raises(V.VlasovError) as e:
            s.sync()
        assert e.value.code == V.ETIMEOUT
        s.sync()                                      # the flag was cleared by the report
        # the path through get_f reports it as well
        s.test_expire_wait(1_000)
        with pytest.raises(V.VlasovError) as e:
            s.get_f()
        assert e.value.code == V.ETIMEOUT
        # the same handle keeps stepping and matches a fresh handle run from the same state
        s.set_f(f0)
        s.step(5)
        fa, ma = s.get_f(), s.moments()
    with V.Sim.from_workload(w, precision="fx64") as t:
        t.set_f(f0)
        t.step(5)
        fb, mb = t.get_f(), t.moments()
    assert np.array_equal(fa, fb)
    assert np.array_equal(ma, mb)


def test_expire_wait_limits_are_checked():
    w = I.HMF_256.resized(64)
    with V.Sim.from_workload(w, precision="f32") as s:
        for bad in (0, 999, 3_000_000_000):
            with pytest.raises(V.VlasovError) as e:
                s.test_expire_wait(bad)
            assert e.value.code == V.EINVAL
