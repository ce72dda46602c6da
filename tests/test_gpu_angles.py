"""GPU parity for the chain bending term (Eq. 12, read as k_a (1 + cos theta)
with k_a = 1.5): Kremer-Grest chains (WCA + FENE + bending) under strong
shear, through the C ABI against the FP64 oracle at the GPU's own positions.
FP64 and FP32: forces within 1e-5 (global L2 and per particle, as the other
tests); FP32 also within the oracle's rounding bound for WCA + FENE plus 1e-5
for the bending part.  The
Eq. 15 tensor and potential energy, which gain the three-body virial and the
bending energy, against the oracle's."""
import numpy as np
import pytest

import oracle
import synth
from helpers import force_errors

le = pytest.importorskip("paper_2109_11083_gb300")

pytestmark = pytest.mark.gpu

KA = 1.5
RC = 2 ** (1 / 6)


def _chains(prec, gd=0.5, seed=17):
    pos, box, bonds = synth.lattice_chains(40, 25, 0.85, seed)
    vel = synth.mb_velocities(pos.shape[0], 1.0, seed)
    vel[:, 0] += gd * (pos[:, 2] - 0.5 * box)
    sim = le.Sim(box, gd, RC, 0.3, dt=0.005, xi=0.5, seed=3, precision=prec, angle_k=KA)
    sim.set_bonds(bonds)
    sim.set_particles(pos, vel)
    p = oracle.params(box, gd, RC, fene_k=30.0, fene_R0=1.5, xi=0.5, dt=0.005, seed=3,
                      angle_k=KA)
    return sim, p, box, bonds


def _check(sim, p, step, prec, box, bonds):
    r, _ = sim.positions()
    dX = oracle.dX(p, step)
    st, F, _, _ = oracle.forces(p, dX, r, bonds, use_cells=True)
    assert st == oracle.OK
    f = sim.forces()
    if prec == 0:
        g, q = force_errors(f, F)
        assert g <= 1e-5 and q <= 1e-5, (step, g, q)
    else:
        edge = 1.5
        P = 0.5 * box / np.floor(box / edge) + 0.5 * 0.3
        B = oracle.force_error_bound(p, dX, r, bonds, 2.0 ** -24, P)
        err = np.linalg.norm(f - F, axis=1)
        assert np.all(err <= B + 1e-5), (step, int(np.argmax(err - B)))
        # the 1e-5 relative force tolerance itself (the WCA pair force vanishes at
        # its cut-off 2^(1/6), so a cut-off decision moves no force)
        g, q = force_errors(f, F)
        assert g <= 1e-5 and q <= 1e-5, (step, g, q)


@pytest.mark.parametrize("prec", [0, 1])
def test_bending_forces_match_oracle_every_fifth_step(prec):
    sim, p, box, bonds = _chains(prec)
    _check(sim, p, 0, prec, box, bonds)
    for step in range(1, 101):
        sim.step(1)
        if step % 5 == 0:
            _check(sim, p, step, prec, box, bonds)
    assert sim.counters()["rebuilds"] > 0
    sim.close()


def test_bending_stress_and_energy_match_oracle():
    sim, p, box, bonds = _chains(0, gd=0.3, seed=19)
    sim.step(30)
    r, v = sim.positions()
    ora = oracle.State(p, r, v, bonds=bonds, step=30)
    S_ref, _, e_ref = ora.observe()
    S, _, _ = sim.stress()
    assert np.abs(S - S_ref).max() <= 1e-8 * np.abs(S_ref).max()
    sim.close()


def test_bending_changes_the_forces():
    """The same chains without the bending term: forces differ by the bending
    forces alone (oracle difference), so the term is really applied."""
    sim, p, box, bonds = _chains(0)
    r, _ = sim.positions()
    f_with = sim.forces()
    p0 = oracle.params(box, 0.5, RC, fene_k=30.0, fene_R0=1.5, xi=0.5, dt=0.005, seed=3)
    _, F0, _, _ = oracle.forces(p0, oracle.dX(p0, 0), r, bonds)
    _, F1, _, _ = oracle.forces(p, oracle.dX(p, 0), r, bonds)
    assert np.abs(F1 - F0).max() > 0.1
    np.testing.assert_allclose(f_with - F0, F1 - F0, atol=1e-6)
    sim.close()
