"""Batched stepping: many uneven boxes advanced by one graph launch give, for
every member, exactly the trajectory of stepping that box alone."""
import numpy as np
import pytest

import synth

le = pytest.importorskip("paper_2109_11083_gb300")

pytestmark = pytest.mark.gpu


def _box(spec, prec, bins=8):
    pos, box = synth.lj_box(spec["n"], spec["rho"], spec["seed"])
    vel = synth.mb_velocities(spec["n"], 1.0, spec["seed"])
    gd = spec["shear_rate"]
    vel[:, 0] += gd * (pos[:, 2] - 0.5 * box)
    sim = le.Sim(box, gd, 2.5, 0.3, seed=spec["seed"], system_id=spec["seed"], precision=prec,
                 profile_bins=bins)
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


def _kg(seed, prec):
    pos, box, bonds = synth.lattice_chains(20, 20, 0.85, seed)
    vel = synth.mb_velocities(pos.shape[0], 1.0, seed)
    vel[:, 0] += 0.2 * (pos[:, 2] - 0.5 * box)
    sim = le.Sim(box, 0.2, 2 ** (1 / 6), 0.3, dt=0.005, xi=0.5, seed=seed, system_id=seed,
                 precision=prec, angle_k=1.5, profile_bins=8)
    sim.set_bonds(bonds)
    sim.set_particles(pos, vel)
    return sim


def _dpd(seed, prec):
    pos, box = synth.lj_box(1500, 0.8442, seed)
    vel = synth.mb_velocities(1500, 1.0, seed)
    vel[:, 0] += 0.4 * (pos[:, 2] - 0.5 * box)
    sim = le.Sim(box, 0.4, 2.5, 0.3, seed=seed, system_id=seed, precision=prec, xi=4.5,
                 thermostat=le.LE_THERMO_DPD, profile_bins=8)
    sim.set_particles(pos, vel)
    return sim


def test_mixed_groups_equal_alone_bitwise():
    """Members of different precision, with and without bonds, Langevin and
    DPD, in one batch (several launch groups): each equals its run alone."""
    specs = synth.batched_systems(count=3, nmin=800, nmax=4000, seed=81)

    def make():
        # profile bin counts differ between members of one launch group
        return ([_box(s, p, b) for s, p, b in zip(specs, (1, 0, 1), (8, 8, 40))] +
                [_kg(31, 1), _kg(32, 0), _dpd(33, 1), _dpd(34, 0)])

    alone, mixed = make(), make()
    for a in alone:
        a.step(48)
    with le.Batch() as b:
        for m in mixed:
            b.add(m)
        b.step(48)
    for a, m in zip(alone, mixed):
        ra, va = a.positions()
        rm, vm = m.positions()
        assert np.array_equal(ra, rm) and np.array_equal(va, vm)
        assert np.array_equal(a.forces(), m.forces())
        assert a.stress(instantaneous=False)[1] == m.stress(instantaneous=False)[1]
        assert a.counters()["rebuilds"] == m.counters()["rebuilds"] > 0
        for x, y in zip(a.profiles(), m.profiles()):
            assert np.array_equal(x, y, equal_nan=True)
    for s in alone + mixed:
        s.close()


def test_members_with_one_and_two_sort_passes_equal_alone_bitwise():
    """Boxes small enough for a one-pass radix sort of their cell keys and
    large enough to need two (over 512 cells), in one batch launch."""
    specs = [{"n": n, "rho": 0.8442, "shear_rate": gd, "seed": 400 + k}
             for k, (n, gd) in enumerate([(700, 0.9), (20000, 0.05), (1500, 0.3),
                                          (26000, 0.2)])]
    alone = [_box(s, 1) for s in specs]
    mixed = [_box(s, 1) for s in specs]
    passes = []
    for a in alone:
        c = a.counters()
        ncell = c["cells"][0] * c["cells"][1] * c["cells"][2]
        passes.append(1 if ncell <= 512 else 2)
        a.step(40)
    assert set(passes) == {1, 2}
    with le.Batch() as b:
        for m in mixed:
            b.add(m)
        b.step(40)
    for a, m in zip(alone, mixed):
        ra, va = a.positions()
        rm, vm = m.positions()
        assert np.array_equal(ra, rm) and np.array_equal(va, vm)
        assert a.counters()["rebuilds"] == m.counters()["rebuilds"] > 0
    for s in alone + mixed:
        s.close()


def test_member_with_a_multi_block_count_table_scan_equal_alone_bitwise():
    """A member large enough that its radix passes scan their count tables
    with the three-kernel scan (1.1M particles: 39^3 cells, two passes of
    8 bits, 256 buckets x 269 tiles of 4096 keys > 8 chunks of 4096), batched
    with two small boxes whose tables are scanned in one block."""
    specs = [{"n": 1_100_000, "rho": 0.8442, "shear_rate": 0.5, "seed": 510},
             {"n": 900, "rho": 0.8, "shear_rate": 0.7, "seed": 511},
             {"n": 5000, "rho": 0.75, "shear_rate": 0.02, "seed": 512}]
    alone = [_box(s, 1) for s in specs]
    mixed = [_box(s, 1) for s in specs]
    c = alone[0].counters()
    assert c["cells"][0] * c["cells"][1] * c["cells"][2] > 2 ** 15
    for a in alone:
        a.step(24)
    with le.Batch() as b:
        for m in mixed:
            b.add(m)
        b.step(24)
    for a, m in zip(alone, mixed):
        ra, va = a.positions()
        rm, vm = m.positions()
        assert np.array_equal(ra, rm) and np.array_equal(va, vm)
        assert a.counters()["rebuilds"] == m.counters()["rebuilds"] > 1
    for s in alone + mixed:
        s.close()


def test_batch_of_more_members_than_one_activation_chunk_equal_alone_bitwise():
    """300 small members: the per-step table of rebuilding members is built
    in chunks of 256 members (a running carry across chunks); sampled
    members, including ones past the first chunk, equal the same box alone."""
    specs = synth.batched_systems(count=300, nmin=500, nmax=900, seed=91)
    mixed = [_box(s, 1, bins=4) for s in specs]
    sample = list(range(0, 300, 23)) + [255, 256, 257, 299]
    alone = {k: _box(specs[k], 1, bins=4) for k in sample}
    for a in alone.values():
        a.step(30)
    with le.Batch() as b:
        for m in mixed:
            b.add(m)
        b.step(30)
    for k, a in alone.items():
        ra, va = a.positions()
        rm, vm = mixed[k].positions()
        assert np.array_equal(ra, rm) and np.array_equal(va, vm), k
        assert a.counters()["rebuilds"] == mixed[k].counters()["rebuilds"] > 1
    for s in list(alone.values()) + mixed:
        s.close()


def test_a_member_error_rolls_every_member_back():
    """One member breaks a FENE bond (two bonded beads flying apart): the batch
    call reports it and every member is back at its state before the call."""
    specs = synth.batched_systems(count=3, nmin=800, nmax=2000, seed=17)
    good = [_box(s, 1) for s in specs]
    pos = np.array([[2.0, 2.0, 2.0], [3.0, 2.0, 2.0], [5.0, 5.0, 5.0]])
    vel = np.array([[-30.0, 0, 0], [30.0, 0, 0], [0, 0, 0]])
    bad = le.Sim(10.0, 0.0, 2 ** (1 / 6), 0.3, thermostat=0, dt=0.01, precision=1)
    bad.set_bonds([[0, 1]])
    bad.set_particles(pos, vel)
    with le.Batch() as b:
        for s in good:
            b.add(s)
        b.step(10)
        b.add(bad)
        before = [s.positions() for s in good + [bad]]
        steps0 = [s.counters()["step"] for s in good + [bad]]
        with pytest.raises(le.LEError) as e:
            b.step(50)
        assert e.value.status == 5
        for s, (r0, v0), n0 in zip(good + [bad], before, steps0):
            r1, v1 = s.positions()
            assert np.array_equal(r0, r1) and np.array_equal(v0, v1)
            assert s.counters()["step"] == n0
    for s in good + [bad]:
        s.close()
