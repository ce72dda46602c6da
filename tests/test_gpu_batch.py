"""Batched stepping: many uneven boxes advanced by one graph launch give, for
every member, exactly the trajectory of stepping that box alone."""
import numpy as np
import pytest

import synth

le = pytest.importorskip("paper_2109_11083_gb300")

pytestmark = pytest.mark.gpu


def _box(spec, prec):
    pos, box = synth.lj_box(spec["n"], spec["rho"], spec["seed"])
    vel = synth.mb_velocities(spec["n"], 1.0, spec["seed"])
    gd = spec["shear_rate"]
    vel[:, 0] += gd * (pos[:, 2] - 0.5 * box)
    sim = le.Sim(box, gd, 2.5, 0.3, seed=spec["seed"], system_id=spec["seed"], precision=prec,
                 profile_bins=8)
    sim.set_particles(pos, vel)
    return sim


@pytest.mark.parametrize("prec", [0, 1])
def test_batched_members_equal_alone_bitwise(prec):
    specs = synth.batched_systems(count=6, nmin=500, nmax=6000, seed=77)
    alone = [_box(s, prec) for s in specs]
    mixed = [_box(s, prec) for s in specs]
    for a in alone:
        a.step(70)
    with le.Batch() as b:
        for m in mixed:
            b.add(m)
        b.step(50)
        b.remove(mixed[2])          # membership changes mid-run
        mixed[2].step(20)           # a removed member steps on its own
        b.step(20)
    for a, m in zip(alone, mixed):
        ra, va = a.positions()
        rm, vm = m.positions()
        assert np.array_equal(ra, rm) and np.array_equal(va, vm)
        assert np.array_equal(a.forces(), m.forces())
        assert a.stress(instantaneous=False)[1] == m.stress(instantaneous=False)[1]
        pa, ca = a.velocity_profile()
        pm, cm = m.velocity_profile()
        assert np.array_equal(ca, cm) and np.array_equal(pa, pm)
        assert a.counters()["step"] == m.counters()["step"] == 70
    for s in alone + mixed:
        s.close()


def test_batch_budget_refuses_a_member_beyond_it():
    specs = synth.batched_systems(count=2, nmin=2000, nmax=3000, seed=5)
    sims = [_box(s, 1) for s in specs]
    p = le.le_default_params()
    p.precision = 1
    need = le.le_estimate_device_bytes(sims[0].box, sims[0].shear_rate, 2.5, 0.3, p,
                                       specs[0]["n"])
    assert need > 0
    with le.Batch(budget_bytes=int(need * 1.5)) as b:
        b.add(sims[0])
        with pytest.raises(le.LEError) as e:
            b.add(sims[1])
        assert e.value.status == 3
    for s in sims:
        s.close()
