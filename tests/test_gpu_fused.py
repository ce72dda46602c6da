"""Inside a call of several steps (FP32 without DPD) the pair kernel of each
step but the last also runs the next step's half kick and drift, writing the
drifted fixed-point positions to a second array.  The same steps taken one
call at a time have a drift launch of their own every step.  Both forms must
give the same bits: positions, velocities, forces, the running xz stress,
temperature and profiles, and the list-build count."""
import numpy as np
import pytest

import synth

le = pytest.importorskip("paper_2109_11083_gb300")

pytestmark = pytest.mark.gpu


def _observables(sim):
    r, v = sim.positions()
    _, xz, ns = sim.stress(instantaneous=False)
    vx, ty, rho, cnt = sim.profiles()
    return (r, v, sim.forces(), xz, ns, sim.temperature(), vx, ty, rho, cnt,
            sim.counters()["rebuilds"])


def _assert_same(a, b):
    for x, y in zip(_observables(a), _observables(b)):
        assert np.array_equal(np.asarray(x), np.asarray(y))


def _pair(pos, vel, box, gd, rc, bonds=None, **kw):
    sims = []
    for _ in range(2):
        s = le.Sim(box, gd, rc, 0.3, seed=3, precision=le.LE_FP32, profile_bins=10, **kw)
        if bonds is not None:
            s.set_bonds(bonds)
        s.set_particles(pos, vel)
        sims.append(s)
    return sims


@pytest.mark.parametrize("gd,thermostat", [(0.05, 1), (1.0, 1), (0.5, 2)])
def test_fused_calls_equal_single_steps_lj(gd, thermostat):
    pos, box = synth.lj_box(3000, 0.8442, 5)
    vel = synth.mb_velocities(3000, 1.0, 5)
    vel[:, 0] += gd * (pos[:, 2] - 0.5 * box)
    a, b = _pair(pos, vel, box, gd, 2.5, thermostat=thermostat)
    a.step(100)                 # six 16-step graphs and four single steps
    for _ in range(100):
        b.step(1)               # a drift launch in every step
    _assert_same(a, b)
    assert a.counters()["rebuilds"] > 3   # list builds inside fused calls


def test_fused_calls_equal_single_steps_chains():
    """FENE chains (bond separations read through the fixed-point copy)."""
    pos, box, bonds = synth.lattice_chains(40, 25, 0.85, 13)
    gd = 0.5
    vel = synth.mb_velocities(pos.shape[0], 1.0, 13)
    vel[:, 0] += gd * (pos[:, 2] - 0.5 * box)
    a, b = _pair(pos, vel, box, gd, 2.0 ** (1.0 / 6.0), bonds=bonds, fene_k=30.0)
    a.step(64)
    for _ in range(64):
        b.step(1)
    _assert_same(a, b)


def test_fused_call_rolls_back_on_error():
    """A bond that breaks inside a multi-step FP32 call (fused pair and drift
    launches, the fixed-point copies swapped every step) rolls the whole call
    back: positions, velocities, forces and the step count are those before
    the call, and the same call fails again the same way."""
    pos = np.array([[2.0, 2.0, 2.0], [3.0, 2.0, 2.0], [5.0, 5.0, 5.0], [7.0, 7.0, 7.0]])
    # the bond stretches 0.2 a step at first: past R0 = 1.5 a few steps in
    vel = np.array([[-10.0, 0, 0], [10.0, 0, 0], [0, 0, 0], [0.5, 0, 0]])
    sim = le.Sim(10.0, 0.1, 2 ** (1 / 6), 0.3, thermostat=0, dt=0.01, precision=le.LE_FP32)
    sim.set_bonds([[0, 1]])
    sim.set_particles(pos, vel)
    r0, v0 = sim.positions()
    f0 = sim.forces()
    for _ in range(2):
        with pytest.raises(le.LEError) as e:
            sim.step(50)
        assert e.value.status == 5
        r1, v1 = sim.positions()
        assert np.array_equal(r0, r1) and np.array_equal(v0, v1)
        assert np.array_equal(f0, sim.forces())
        assert sim.counters()["step"] == 0
    sim.close()
