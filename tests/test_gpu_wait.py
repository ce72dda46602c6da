"""Failure detection without a fault: the bounded mbarrier wait that the pair
kernel uses for its bulk copies of list rows, run on a barrier that nothing
completes, gives up (about a second) and comes back as LE_ERR_TIMEOUT, and the
device keeps working afterwards."""
import numpy as np
import pytest

import synth

le = pytest.importorskip("paper_2109_11083_gb300")

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_the_device_stays_usable():
    st, ms = le.le_wait_selftest()
    assert st == 8                     # LE_ERR_TIMEOUT: the wait ended, as designed
    assert 1.0 < ms < 20000.0          # it waited, and it did end
    pos, box = synth.lj_box(500, 0.8442, 3)
    vel = synth.mb_velocities(500, 1.0, 3)
    sim = le.Sim(box, 0.1, 2.5, 0.3, seed=3, precision=le.LE_FP32)
    sim.set_particles(pos, vel)
    sim.step(20)
    r, v = sim.positions()
    assert np.isfinite(r).all() and np.isfinite(v).all()
    assert sim.counters()["step"] == 20
    sim.close()
