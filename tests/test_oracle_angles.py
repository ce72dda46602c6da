"""Pins for the oracle's bending term (Eq. 12, read as the cosine potential
k_a (1 + cos theta) with its minimum at the stated 180 degrees): energy
gradient by finite differences, a right-angle closed form, a straight chain,
zero net torque, and a chain across the sheared top face against the same
chain unwrapped in a large box.  LJ and FENE are off (eps = 0, k = 0) so
each test sees the angle term alone.  No GPU is used here."""
import numpy as np

import oracle

KA = 1.5


def _params(box, gd=0.0, dt=0.005):
    return oracle.params(box, gd, 1.0, eps=0.0, fene_k=0.0, angle_k=KA, dt=dt)


def _forces(p, dX, pos, bonds):
    st, F, W, e = oracle.forces(p, dX, np.asarray(pos, float), np.asarray(bonds), use_cells=False)
    assert st == oracle.OK
    return F, W, e


def _chains(rng, nchains, nbeads, box):
    pos, bonds = [], []
    for c in range(nchains):
        r = rng.uniform(0.3 * box, 0.7 * box, 3)
        for b in range(nbeads):
            if b:
                step = rng.normal(size=3)
                r = r + 0.97 * step / np.linalg.norm(step)
                bonds.append((len(pos) - 1, len(pos)))
            pos.append(r.copy())
    return np.array(pos), np.array(bonds, dtype=np.int32)


def test_forces_are_minus_the_energy_gradient():
    rng = np.random.default_rng(3)
    box = 20.0
    pos, bonds = _chains(rng, 3, 6, box)
    p = _params(box)
    F, _, _ = _forces(p, 0.0, pos, bonds)
    h = 1e-6
    for i in (0, 4, 9, 17):
        for a in range(3):
            up, dn = pos.copy(), pos.copy()
            up[i, a] += h
            dn[i, a] -= h
            de = _forces(p, 0.0, up, bonds)[2] - _forces(p, 0.0, dn, bonds)[2]
            assert abs(-de / (2 * h) - F[i, a]) < 1e-7


def test_right_angle_closed_form_and_straight_chain():
    box = 10.0
    j = np.array([5.0, 5.0, 5.0])
    pos = np.array([j + [1.0, 0, 0], j, j + [0, 1.4, 0]])
    bonds = np.array([[0, 1], [1, 2]], dtype=np.int32)
    F, _, e = _forces(_params(box), 0.0, pos, bonds)
    # cos theta = 0: F_i = -k_a c^/|a|, F_k = -k_a a^/|c|
    np.testing.assert_allclose(F[0], [0, -KA, 0], atol=1e-14)
    np.testing.assert_allclose(F[2], [-KA / 1.4, 0, 0], atol=1e-14)
    np.testing.assert_allclose(F[1], [KA / 1.4, KA, 0], atol=1e-14)
    assert abs(e - KA) < 1e-14
    straight = np.array([j - [0.9, 0, 0], j, j + [1.1, 0, 0]])
    F, _, e = _forces(_params(box), 0.0, straight, bonds)
    assert np.abs(F).max() < 1e-14 and abs(e) < 1e-14


def test_no_net_force_or_torque():
    rng = np.random.default_rng(5)
    box = 30.0
    pos, bonds = _chains(rng, 2, 8, box)
    F, _, _ = _forces(_params(box), 0.0, pos, bonds)
    assert np.abs(F.sum(axis=0)).max() < 1e-12
    torque = np.cross(pos - pos.mean(axis=0), F).sum(axis=0)
    assert np.abs(torque).max() < 1e-12


def test_chain_across_the_sheared_face_equals_the_unwrapped_chain():
    """Beads placed by the LE wrap (through the top face z -= Lz, x -= dX)
    feel the same bending forces as the unwrapped chain in a box so large
    that no image is involved."""
    rng = np.random.default_rng(7)
    box, dX = 8.0, 3.1
    start = np.array([2.0, 4.0, box - 1.2])
    pos = [start]
    for b in range(5):
        step = rng.normal(size=3)
        step[2] = abs(step[2]) + 0.5            # climb through the top face
        pos.append(pos[-1] + 0.97 * step / np.linalg.norm(step))
    pos = np.array(pos)
    bonds = np.array([[b, b + 1] for b in range(5)], dtype=np.int32)
    wrapped = pos.copy()
    up = wrapped[:, 2] >= box
    wrapped[up, 2] -= box
    wrapped[up, 0] -= dX
    wrapped[:, 0] = np.mod(wrapped[:, 0], box)
    wrapped[:, 1] = np.mod(wrapped[:, 1], box)
    assert up.any() and not up.all()
    F_le, _, e_le = _forces(_params(box), dX, wrapped, bonds)
    F_free, _, e_free = _forces(_params(1000.0), 0.0, pos + 400.0, bonds)
    np.testing.assert_allclose(F_le, F_free, atol=1e-12)
    assert abs(e_le - e_free) < 1e-12
