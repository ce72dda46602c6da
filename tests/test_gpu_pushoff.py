"""The Kremer-Grest initial condition of the melt workload, built as stated:
freely jointed random walks of bond length 0.97 (Sec. 2.4), a force-capped
push-off (le_params force_cap, FP64), then an uncapped melt.

- Capped forces of overlapping random-walk chains (WCA + FENE) against the
  oracle's capped forces: relative 1e-5, as every FP64 force.
- The push-off removes the overlaps (no two non-bonded beads closer than 0.8)
  with every bond intact, and the melt then steps without a cap in FP32.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import force_errors, le_delta

le = pytest.importorskip("paper_2109_11083_gb300")
from paper_2109_11083_gb300 import prepare  # noqa: E402

pytestmark = pytest.mark.gpu

RC = 2 ** (1 / 6)


def _min_nonbonded(pos, box, bonds):
    from scipy.spatial import cKDTree
    t = cKDTree(np.mod(pos, box), boxsize=box)
    pairs = t.query_pairs(0.9, output_type="ndarray")
    bonded = {(min(a, b), max(a, b)) for a, b in np.asarray(bonds)}
    d = [np.linalg.norm(le_delta(pos[[a]], pos[[b]], box, 0.0)) for a, b in pairs
         if (min(a, b), max(a, b)) not in bonded]
    return min(d) if d else 0.9


def test_capped_forces_match_oracle():
    pos, box, bonds = synth.random_walk_chains(40, 30, 0.85, 7)
    cap = 30.0
    sim = le.Sim(box, 0.0, RC, 0.3, precision=0, force_cap=cap, thermostat=0, sample_every=0)
    sim.set_bonds(bonds)
    sim.set_particles(pos, np.zeros_like(pos))
    p = oracle.params(box, 0.0, RC, fene_k=30.0, fene_R0=1.5, force_cap=cap)
    r, _ = sim.positions()
    st, F, _, _ = oracle.forces(p, 0.0, r, bonds)
    assert st == oracle.OK
    g, q = force_errors(sim.forces(), F)
    assert g <= 1e-5 and q <= 1e-5, (g, q)
    # the cap binds: some pair of the random walks overlaps
    _, F0, _, _ = oracle.forces(oracle.params(box, 0.0, RC, fene_k=30.0, fene_R0=1.5), 0.0, r, bonds)
    assert np.abs(F0).max() > 10 * cap
    sim.close()


def test_fp32_rejects_a_force_cap():
    with pytest.raises(le.LEError) as e:
        le.Sim(10.0, 0.0, RC, 0.3, precision=1, force_cap=10.0)
    assert e.value.status == 1


def test_push_off_then_uncapped_melt():
    pos, box, bonds = synth.random_walk_chains(50, 40, 0.85, 11)
    assert _min_nonbonded(pos, box, bonds) < 0.3          # the walks overlap
    pos2, vel2 = prepare.push_off(pos, box, bonds, seed=3)
    dmin = _min_nonbonded(pos2, box, bonds)
    b = le_delta(pos2[bonds[:, 0]], pos2[bonds[:, 1]], box, 0.0)
    lb = np.linalg.norm(b, axis=1)
    print(f"\npush-off: closest non-bonded pair {dmin:.3f}, bonds {lb.min():.3f}..{lb.max():.3f}")
    assert dmin > 0.8 and lb.max() < 1.3
    sim = le.Sim(box, 0.0, RC, 0.3, precision=1, dt=0.005, xi=0.5, seed=5)
    sim.set_bonds(bonds)
    sim.set_particles(pos2, vel2)
    sim.step(2000)
    assert 0.9 < sim.temperature() < 1.1
    sim.close()
