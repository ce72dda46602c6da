"""Pins for the oracle's DPD thermostat (Eqs. 6-8, read as the textbook
fluctuation-dissipation form with the paper's sqrt(24 kT xi) theta noise,
divided by sqrt(dt)).  Each test ties it to a library routine, an invariant
or a symmetry, not to itself.  No GPU is used here."""
import numpy as np
import pytest

import oracle
import synth


def _dpd(n, gd, seed, xi=4.5, kT=1.0, rho=0.8442):
    pos, box = synth.lj_box(n, rho, seed)
    vel = synth.mb_velocities(n, kT, seed)
    vel[:, 0] += gd * (pos[:, 2] - 0.5 * box)
    p = oracle.params(box, gd, 2.5, xi=xi, kT=kT, thermostat=3, seed=11, system=2)
    return p, pos, vel, box


def test_pair_noise_is_the_library_philox_and_symmetric():
    """theta_ij is the first output word of Philox4x64-10 at counter
    (step, min id, max id, 1) with key (seed, system) -- checked against
    numpy's implementation of the generator -- and the same for (i, j) and
    (j, i)."""
    p = oracle.params(10.0, 0.0, 2.5, seed=2109, system=7)
    for step, a, b in [(0, 1, 2), (17, 900, 3), (2 ** 40, 5, 123456)]:
        lo, hi = min(a, b), max(a, b)
        # numpy advances the counter before each block: start one below
        bg = np.random.Philox(key=np.array([2109, 7], dtype=np.uint64),
                              counter=np.array([step - 1 if step else 2 ** 64 - 1,
                                                lo if step else lo - 1, hi, 1], dtype=np.uint64))
        word = int(bg.random_raw())
        want = (word >> 11) * 2.0 ** -53 - 0.5
        assert oracle.pair_uniform(p, step, a, b) == want
        assert oracle.pair_uniform(p, step, b, a) == want


@pytest.mark.parametrize("gd", [0.0, 0.7])
def test_dpd_forces_are_pairwise(gd):
    """F_ji = -F_ij for every pair, across the sheared face too (the image's
    velocity is shifted consistently), so the thermostat forces sum to zero."""
    p, pos, vel, _ = _dpd(2000, gd, 4)
    Fc, Ft = oracle.thermostat_forces(p, 3, pos, vel)
    dpd = Ft - Fc
    assert np.abs(dpd).max() > 1.0
    assert np.abs(dpd.sum(axis=0)).max() < 1e-10 * np.abs(dpd).sum()


def test_dpd_is_galilean_invariant():
    p, pos, vel, _ = _dpd(1000, 0.3, 5)
    _, F1 = oracle.thermostat_forces(p, 2, pos, vel)
    _, F2 = oracle.thermostat_forces(p, 2, pos, vel + np.array([0.7, -1.3, 0.4]))
    np.testing.assert_allclose(F2, F1, atol=1e-12, rtol=0)


def test_linear_flow_on_a_lattice_dissipates_nothing():
    """A perfect fcc lattice moving with the linear profile v = shear (z - Lz/2)
    e_x, no noise (kT = 0): every pair +d has a partner -d with the same
    relative velocity along its bond, so each particle's dissipative force
    cancels -- also next to the faces, where the partner is an image whose
    velocity is shifted by the shear across the box.  (A wrong sign of that
    shift leaves the face layers with forces of order xi shear Lz.)"""
    k = 8
    a = (4 / 0.8442) ** (1 / 3)
    base = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    g = np.array([[i, j, l] for i in range(k) for j in range(k) for l in range(k)], float)
    pos = ((g[:, None, :] + base[None, :, :]).reshape(-1, 3) + 0.25) * a
    box = k * a
    gd = 0.6
    vel = np.zeros_like(pos)
    vel[:, 0] = gd * (pos[:, 2] - 0.5 * box)
    p = oracle.params(box, gd, 2.5, xi=4.5, kT=0.0, thermostat=3)
    Fc, Ft = oracle.thermostat_forces(p, 0, pos, vel)
    near_face = (pos[:, 2] < 2.5) | (pos[:, 2] > box - 2.5)
    assert near_face.any()
    assert np.abs(Ft - Fc).max() < 1e-10


def test_dpd_thermalizes_to_kT():
    """With no shear the fluctuation-dissipation relation holds the peculiar
    temperature at kT (to the discretisation and sampling error)."""
    p, pos, vel, _ = _dpd(1500, 0.0, 6, xi=4.5, kT=1.0)
    s = oracle.State(p, pos, vel)
    assert s.run(300) == oracle.OK
    T = []
    for _ in range(10):
        assert s.run(20) == oracle.OK
        T.append(s.observe()[1])
    assert abs(np.mean(T) - 1.0) < 0.05, T
