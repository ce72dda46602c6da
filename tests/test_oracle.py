"""Pins for the FP64 CPU oracle: each test ties part of it to something other
than itself (a library routine, a closed form, an invariant of the equations
or brute force on tiny inputs).  No GPU is used here."""
import math

import numpy as np
import pytest
from scipy.spatial import cKDTree

import oracle
import synth
from oracle import brute
from helpers import shear_affine


def jittered_lattice(n, rho, seed, amp=0.05):
    pos, box = synth.lj_box(n, rho, seed)
    pos = pos + np.random.default_rng(seed + 1).uniform(-amp, amp, size=pos.shape)
    return np.mod(pos, box), box


# --------------------------------------------------------------------------- RNG
@pytest.mark.parametrize("ctr,key", [
    ((0, 0, 0, 0), (0, 0)),
    ((5, 17, 0, 0), (2109, 3)),
    ((2**64 - 1, 2**63 + 11, 7, 2**40), (2**64 - 5, 123456789)),
])
def test_philox_matches_numpy_library(ctr, key):
    """Philox4x64-10 agrees with numpy's implementation of the same published
    generator.  numpy advances its counter before each block, so a generator
    started at counter c-1 yields the block of counter c first."""
    start = np.array(ctr, dtype=np.uint64)
    # counter c-1 with borrow across the 4 x 64-bit words
    words = [int(x) for x in ctr]
    for w in range(4):
        if words[w] > 0:
            words[w] -= 1
            break
        words[w] = 2**64 - 1
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                          counter=np.array(words, dtype=np.uint64))
    expect = bg.random_raw(4)
    got = oracle.philox4x64(start, key)
    assert np.array_equal(got, expect)


def test_noise_is_uniform_with_the_stated_moments():
    """U(-1/2, 1/2): mean 0 and variance 1/12 (so the random force has
    variance 2 xi kT m / dt), independent components and particles."""
    p = oracle.params(10.0, 0.0, 2.5, seed=99, system=4)
    u = np.array([oracle.noise(p, step, gid) for step in range(40) for gid in range(1000)])
    n = u.size
    assert u.min() >= -0.5 and u.max() < 0.5
    assert abs(u.mean()) < 5 * math.sqrt(1 / 12 / n)
    assert abs(u.var() - 1 / 12) < 5 * math.sqrt(1 / 180 / n)
    c = np.corrcoef(u.T)
    assert np.all(np.abs(c - np.eye(3)) < 5 / math.sqrt(u.shape[0]))
    # the 3 components differ between consecutive particles and steps
    assert not np.allclose(oracle.noise(p, 1, 0), oracle.noise(p, 1, 1))
    assert not np.allclose(oracle.noise(p, 1, 0), oracle.noise(p, 2, 0))
    # a different system id gives a different stream (batched systems)
    q = oracle.params(10.0, 0.0, 2.5, seed=99, system=5)
    assert not np.allclose(oracle.noise(p, 1, 0), oracle.noise(q, 1, 0))


# ---------------------------------------------------------------------- Eq. 4 dX
def test_image_offset_closed_form():
    """dX = gamma_dot * Lz * t reduced into [0, Lx) (Eq. 4 / Fig. 1)."""
    p = oracle.params([4.0, 5.0, 10.0], 0.1, 1.0, dt=0.5)
    assert oracle.dX(p, 0) == 0.0
    assert oracle.dX(p, 3) == pytest.approx(1.5, abs=1e-15)      # 0.1*10*1.5
    assert oracle.dX(p, 10) == pytest.approx(1.0, abs=1e-14)     # 5.0 mod 4
    assert oracle.dX(p, 8) == pytest.approx(0.0, abs=1e-14)      # one full Lx
    q = oracle.params([4.0, 5.0, 10.0], -0.1, 1.0, dt=0.5)
    assert oracle.dX(q, 3) == pytest.approx(2.5, abs=1e-14)      # -1.5 mod 4
    for n in range(0, 2000, 37):
        assert 0.0 <= oracle.dX(p, n) < 4.0


# -------------------------------------------------------------- forces vs images
@pytest.mark.parametrize("use_cells", [False, True])
@pytest.mark.parametrize("frac", [0.0, 0.37, 0.5, 1.0 - 1e-12])
def test_forces_match_image_enumeration(use_cells, frac):
    """LE minimum-image forces (LJ, Eq. 9) equal the sum over explicitly
    enumerated sheared images, at several offsets dX."""
    pos, box = jittered_lattice(256, 0.6, seed=11, amp=0.2)
    L = np.array([box * 1.1, box, box * 0.95])
    pos = pos * (L / box)
    dx = frac * L[0]
    p = oracle.params(L, 0.1, 2.5)
    st, F, W, _ = oracle.forces(p, dx, pos, use_cells=use_cells)
    assert st == oracle.OK
    Fb, Wb, hits = brute.image_forces(pos, L, dx, 2.5)
    assert hits > 1000
    scale = np.abs(Fb).max()
    assert np.abs(F - Fb).max() <= 1e-12 * scale
    assert np.abs(W - Wb).max() <= 1e-12 * np.abs(Wb).max()


def test_cell_mode_equals_all_pairs_on_a_larger_box():
    pos, box = jittered_lattice(2048, 0.8442, seed=5, amp=0.1)
    p = oracle.params(box, 0.1, 2.5)
    for frac in (0.0, 0.213, 0.999):
        _, F0, W0, e0 = oracle.forces(p, frac * box, pos, use_cells=False)
        _, F1, W1, e1 = oracle.forces(p, frac * box, pos, use_cells=True)
        assert np.abs(F0 - F1).max() <= 1e-12 * np.abs(F0).max()
        assert np.abs(W0 - W1).max() <= 1e-12 * np.abs(W0).max()
        assert e0 == pytest.approx(e1, rel=1e-12)


def test_two_particles_across_the_shear_plane():
    """A near the top face, B near the bottom face.  The image box above is
    displaced by +dX, so B's image above sits at (x_B + dX, y, z_B + Lz) and
    the separation is known in closed form: d = (-delta, 0, -(a + b))."""
    L = np.array([12.0, 10.0, 11.0])
    dX, x0, y, a, b, delta = 4.3, 2.0, 5.0, 0.4, 0.55, 0.3
    A = np.array([x0, y, L[2] - a])
    B = np.array([np.mod(x0 + delta - dX, L[0]), y, b])
    p = oracle.params(L, 0.1, 2.5, lj_shift=0)
    d = oracle.min_image(p, dX, A, B)
    assert np.allclose(d, [-delta, 0.0, -(a + b)], atol=1e-14)
    r = math.hypot(delta, a + b)
    f_textbook = 24.0 * (2.0 * r ** -14 - r ** -8)            # eps = sigma = 1
    st, F, W, e = oracle.forces(p, dX, np.stack([A, B]), use_cells=False)
    assert np.allclose(F[0], f_textbook * np.array([-delta, 0.0, -(a + b)]), rtol=1e-13)
    assert np.allclose(F[1], -F[0], rtol=1e-13)
    assert e == pytest.approx(4.0 * (r ** -12 - r ** -6), rel=1e-13)
    # with dX ignored the pair would be far apart in x: the offset matters
    _, F_wrong, _, _ = oracle.forces(p, 0.0, np.stack([A, B]), use_cells=False)
    assert not np.allclose(F_wrong, F)


def test_zero_offset_reduces_to_plain_periodic_boundaries():
    """At dX = 0 (no shear, or a whole number of Lx) the LE system is the
    ordinary periodic one: compare with scipy's periodic KD-tree pair search."""
    pos, box = jittered_lattice(864, 0.8442, seed=3, amp=0.15)
    p = oracle.params(box, 0.0, 2.5)
    _, F, _, _ = oracle.forces(p, 0.0, pos)
    tree = cKDTree(pos, boxsize=box)
    pairs = tree.query_pairs(2.5, output_type="ndarray")
    d = pos[pairs[:, 0]] - pos[pairs[:, 1]]
    d -= box * np.rint(d / box)
    r2 = np.sum(d * d, axis=1)
    keep = r2 < 2.5 ** 2
    pairs, d, r2 = pairs[keep], d[keep], r2[keep]
    fr = brute.lj_f_over_r(r2)
    Fk = np.zeros_like(pos)
    np.add.at(Fk, pairs[:, 0], fr[:, None] * d)
    np.add.at(Fk, pairs[:, 1], -fr[:, None] * d)
    assert np.abs(F - Fk).max() <= 1e-12 * np.abs(Fk).max()
    # an offset of exactly Lx is the same lattice of images
    _, F_lx, _, _ = oracle.forces(p, box, pos)
    assert np.abs(F - F_lx).max() <= 1e-12 * np.abs(F).max()
    # and an offset of dX + Lx equals dX
    _, Fa, _, _ = oracle.forces(p, 0.3 * box, pos)
    _, Fb, _, _ = oracle.forces(p, 1.3 * box, pos)
    assert np.abs(Fa - Fb).max() <= 1e-12 * np.abs(Fa).max()


def kg_chains_small(seed=7, frac=0.0):
    """24 chains of 20 beads, affinely sheared onto the image lattice of
    offset frac*Lx so that bonds through the top/bottom face stay intact."""
    pos, box, bonds = synth.lattice_chains(24, 20, 0.85, seed)
    return shear_affine(pos, box, frac * box), box, bonds


def test_newton_third_law_with_fene_across_the_shear_plane():
    for frac in (0.0, 0.1, 0.25):
        pos, box, bonds = kg_chains_small(frac=frac)
        p = oracle.params(box, 0.3, 2 ** (1 / 6), fene_k=30.0, fene_R0=1.5)
        st, F, _, _ = oracle.forces(p, frac * box, pos, bonds)
        assert st == oracle.OK
        assert np.abs(F.sum(axis=0)).max() <= 1e-12 * np.abs(F).sum()


def test_fene_force_is_the_gradient_of_eq11():
    """Two bonded beads: the force equals -dV/dr of Eq. 11 (central difference)."""
    L = 10.0
    p = oracle.params(L, 0.0, 2 ** (1 / 6), eps=0.0, fene_k=30.0, fene_R0=1.5)
    for r in (0.5, 0.97, 1.3, 1.45):
        A = np.array([[1.0, 1.0, 1.0], [1.0 + r, 1.0, 1.0]])
        st, F, _, e = oracle.forces(p, 0.0, A, [[0, 1]])
        h = 1e-6
        Vp = -0.5 * 30 * 1.5 ** 2 * math.log(1 - ((r + h) / 1.5) ** 2)
        Vm = -0.5 * 30 * 1.5 ** 2 * math.log(1 - ((r - h) / 1.5) ** 2)
        assert F[1, 0] == pytest.approx(-(Vp - Vm) / (2 * h), rel=1e-7)
        assert F[0, 0] == pytest.approx(-F[1, 0], rel=1e-14)


def test_fene_reports_a_broken_bond():
    p = oracle.params(10.0, 0.0, 2 ** (1 / 6), fene_k=30.0, fene_R0=1.5)
    A = np.array([[1.0, 1.0, 1.0], [2.6, 1.0, 1.0]])
    st, _, _, _ = oracle.forces(p, 0.0, A, [[0, 1]])
    assert st == oracle.BOND_BROKEN


@pytest.mark.parametrize("with_bonds", [0, 1, 2])
def test_virial_is_minus_the_shear_strain_derivative_of_the_energy(with_bonds):
    """Affine shear x -> x + e z maps every separation d to d + e d_z e_x,
    including pairs across the shear plane once dX -> dX + e Lz.  Hence
    sum_{i<j} d_z F_x = -dU/de: this pins the virial part of Eq. 15 and the
    sign of the image offset together.  with_bonds = 2 adds the bending term
    of Eq. 12, whose three-body virial a (x) F_i + c (x) F_k is pinned the
    same way."""
    if with_bonds:
        pos, box, bonds = kg_chains_small(seed=9, frac=0.15)
        p = oracle.params(box, 0.2, 2 ** (1 / 6), fene_k=30.0, fene_R0=1.5, lj_shift=1,
                          angle_k=1.5 if with_bonds == 2 else 0.0)
    else:
        pos, box = jittered_lattice(500, 0.8442, seed=21, amp=0.1)
        bonds = None
        p = oracle.params(box, 0.2, 2.5, lj_shift=1)
    dX0 = (0.15 if with_bonds else 0.37) * box
    _, _, W, _ = oracle.forces(p, dX0, pos, bonds)
    h = 1e-6

    def energy(e):
        q = pos.copy()
        q[:, 0] += e * q[:, 2]
        return oracle.forces(p, dX0 + e * box, q, bonds)[3]

    dU = (energy(h) - energy(-h)) / (2 * h)
    assert W[2, 0] == pytest.approx(-dU, rel=2e-6, abs=1e-6)
    assert W[0, 2] == pytest.approx(W[2, 0], rel=1e-12)


# ------------------------------------------------------------------ integration
def lj_state(n, rho, seed, shear, xi, thermostat, kT=1.0, dt=0.005, use_cells=True,
             nbins=20, lab=True):
    pos, box = synth.lj_box(n, rho, seed)
    vel = synth.mb_velocities(n, kT, seed)
    p = oracle.params(box, shear, 2.5, xi=xi, kT=kT, dt=dt, thermostat=thermostat,
                      seed=seed, nbins=nbins)
    if lab:
        vel[:, 0] += shear * (pos[:, 2] - 0.5 * box)
    return oracle.State(p, pos, vel, use_cells=use_cells), box


def total_energy(s):
    _, _, e = s.observe()
    return e + 0.5 * float(np.sum(s.vel * s.vel))


def test_energy_is_conserved_without_shear_or_thermostat():
    s, _ = lj_state(256, 0.8442, 1, 0.0, 0.0, 0, use_cells=False)
    e0 = total_energy(s)
    drift = []
    for _ in range(10):
        assert s.run(100) == oracle.OK
        drift.append(abs(total_energy(s) - e0) / abs(e0))
    assert max(drift) < 1e-4
    assert np.abs(s.vel.sum(axis=0)).max() < 1e-10


def test_momentum_plus_crossing_jumps_is_conserved_under_shear():
    """With xi = 0 the forces conserve momentum; each crossing through the top
    face lowers vx by gamma_dot*Lz (the velocity jump), so
    P_x + m*gamma_dot*Lz*(net upward crossings) stays constant."""
    s, box = lj_state(500, 0.8442, 2, 1.0, 0.0, 0, use_cells=False)
    P0 = s.vel.sum(axis=0).copy()
    assert s.run(400) == oracle.OK
    assert np.abs(s.zimg).sum() > 0
    P = s.vel.sum(axis=0)
    P[0] += 1.0 * box * s.zimg.sum()
    assert np.abs(P - P0).max() < 1e-9


def test_free_particle_stays_on_the_sheared_image_lattice():
    """No forces, no thermostat: the unwrapped motion is a straight line and the
    stored state is its image in box nz = floor(z_u/Lz) at the current offset:
    z = z_u - nz Lz, x = x_u - nz dX(t) (mod Lx), vx = vx_u - nz gamma_dot Lz."""
    L = np.array([6.0, 5.0, 7.0])
    gd, dt = 0.5, 0.01
    p = oracle.params(L, gd, 2.5, eps=0.0, thermostat=0, dt=dt)
    r0 = np.array([[1.0, 2.0, 6.5]])
    v0 = np.array([[0.3, 0.1, 2.7]])
    s = oracle.State(p, r0, v0, use_cells=False)
    for n in range(1, 900):
        s.run(1)
        t = n * dt
        xu, zu = r0[0, 0] + v0[0, 0] * t, r0[0, 2] + v0[0, 2] * t
        nz = math.floor(zu / L[2])
        dx = oracle.dX(p, n)
        assert s.pos[0, 2] == pytest.approx(zu - nz * L[2], abs=1e-11)
        ex = (xu - nz * dx - s.pos[0, 0]) / L[0]
        assert abs(ex - round(ex)) < 1e-11
        assert s.vel[0, 0] == pytest.approx(v0[0, 0] - nz * gd * L[2], abs=1e-12)
        assert s.zimg[0] == nz
    assert s.zimg[0] >= 3


def test_langevin_holds_the_target_temperature_without_shear():
    s, _ = lj_state(256, 0.8442, 4, 0.0, 1.0, 1, kT=1.5, use_cells=False)
    assert s.run(300) == oracle.OK
    temps = []
    for _ in range(120):
        s.run(10)
        temps.append(s.observe()[1])
    assert np.mean(temps) == pytest.approx(1.5, rel=0.04)


@pytest.mark.slow
def test_peculiar_langevin_gives_a_linear_profile_and_positive_viscosity():
    """Sec. 3.1: with the thermostat on peculiar velocities the steady vx(z)
    profile is linear with slope gamma_dot, and eta = <sigma_xz>/gamma_dot > 0
    (Eq. 14)."""
    gd = 0.5
    s, box = lj_state(864, 0.8442, 5, gd, 1.0, 1, nbins=10)
    assert s.run(1000) == oracle.OK
    s.vx_sum[:] = 0
    s.count[:] = 0
    s.samples.nsamples = 0
    s.samples.sxz_sum = 0.0
    assert s.run(2000, sample_every=1) == oracle.OK
    z = (np.arange(10) + 0.5) * box / 10
    slope = np.polyfit(z, s.profile, 1)[0]
    assert slope == pytest.approx(gd, rel=0.05)
    eta = s.samples.sxz_sum / s.samples.nsamples / gd
    assert 0.5 < eta < 10.0


def test_force_cap_limits_each_pair_force_to_the_cap():
    """The push-off cap: an overlapping pair feels exactly the cap along the
    separation; a pair whose Eq. 9 force is below the cap is unchanged."""
    box = 12.0
    cap = 25.0
    pos = np.array([[3.0, 3.0, 3.0], [3.3, 3.4, 3.0], [8.0, 8.0, 8.0], [9.2, 8.0, 8.0]])
    p = oracle.params(box, 0.0, 2.5, force_cap=cap)
    _, F, _, _ = oracle.forces(p, 0.0, pos, use_cells=False)
    d = pos[0] - pos[1]
    assert np.allclose(F[0], cap * d / np.linalg.norm(d), rtol=1e-13)
    assert np.allclose(F[1], -F[0], rtol=1e-13)
    _, F0, _, _ = oracle.forces(oracle.params(box, 0.0, 2.5), 0.0, pos, use_cells=False)
    r = 1.2
    f = 24.0 * (2 * r ** -12 - r ** -6) / r     # Eq. 9 force at r = 1.2 (below the cap)
    assert abs(f) < cap
    assert np.allclose(F[2:], F0[2:], rtol=1e-14)
    assert F0[3, 0] == pytest.approx(f, rel=1e-12)
