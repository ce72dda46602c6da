"""The launch-shape autotuner: the pair and list kernels' threads per block
change no result, so every shape gives the same trajectory bit for bit, and
tuning (which runs and rolls back trial steps) leaves the state untouched."""
import numpy as np
import pytest

import synth

le = pytest.importorskip("paper_2109_11083_gb300")

pytestmark = pytest.mark.gpu


def _sim(n, gd, seed, prec):
    pos, box = synth.lj_box(n, 0.8442, seed)
    vel = synth.mb_velocities(n, 1.0, seed)
    vel[:, 0] += gd * (pos[:, 2] - 0.5 * box)
    sim = le.Sim(box, gd, 2.5, 0.3, seed=seed, precision=prec, profile_bins=8)
    sim.set_particles(pos, vel)
    return sim


def _same(a, b):
    ra, va = a.positions()
    rb, vb = b.positions()
    assert np.array_equal(ra, rb) and np.array_equal(va, vb)
    assert np.array_equal(a.forces(), b.forces())
    assert a.stress(instantaneous=False)[1:] == b.stress(instantaneous=False)[1:]
    pa, pb = a.profiles(), b.profiles()
    for x, y in zip(pa, pb):
        assert np.array_equal(x, y, equal_nan=True)


@pytest.mark.parametrize("prec", [0, 1])
def test_every_launch_shape_gives_the_same_trajectory(prec):
    ref = _sim(3000, 0.3, 12, prec)
    ref.step(45)
    for ft, lt in [(32, 32), (64, 96), (128, 256), (224, 64)]:
        s = _sim(3000, 0.3, 12, prec)
        s.set_launch(ft, lt)
        s.step(45)
        c = s.counters()
        assert (c["force_threads"], c["list_threads"]) == (ft, lt)
        _same(ref, s)
        s.close()
    ref.close()


def test_tune_leaves_the_state_as_it_was():
    a = _sim(5000, 0.5, 14, 1)
    b = _sim(5000, 0.5, 14, 1)
    a.step(20)
    b.step(20)
    f, l, ms = a.tune(32)
    assert f in (128, 256) and l in (64, 128, 256) and ms > 0
    c = a.counters()
    assert c["step"] == 20 and (c["force_threads"], c["list_threads"]) == (f, l)
    a.step(30)
    b.step(30)
    _same(a, b)
    a.close()
    b.close()


def test_tuned_batch_equals_members_alone():
    specs = synth.batched_systems(count=5, nmin=500, nmax=5000, seed=91)

    def box(spec):
        pos, L = synth.lj_box(spec["n"], spec["rho"], spec["seed"])
        vel = synth.mb_velocities(spec["n"], 1.0, spec["seed"])
        gd = spec["shear_rate"]
        vel[:, 0] += gd * (pos[:, 2] - 0.5 * L)
        s = le.Sim(L, gd, 2.5, 0.3, seed=spec["seed"], system_id=spec["seed"], precision=1)
        s.set_particles(pos, vel)
        return s

    alone = [box(s) for s in specs]
    for a in alone:
        a.step(40)
    with le.Batch() as b:
        mixed = [box(s) for s in specs]
        for m in mixed:
            b.add(m)
        f, l, ms = b.tune(16)
        assert f in (128, 256) and l in (64, 128, 256) and ms > 0
        assert all((m.counters()["force_threads"], m.counters()["list_threads"]) == (f, l)
                   for m in mixed)
        b.step(40)
        for a, m in zip(alone, mixed):
            ra, va = a.positions()
            rm, vm = m.positions()
            assert np.array_equal(ra, rm) and np.array_equal(va, vm)
            m.close()
    for a in alone:
        a.close()
