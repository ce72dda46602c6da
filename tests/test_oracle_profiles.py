"""Pins for the oracle's comparison thermostat and z-profiles (Sec. 2.2 and
Sec. 3.1): the Langevin friction on the absolute velocity (the paper's
xi_abs runs), the T_y profile (mean m vy^2 per z bin) and the density
profile.  Each test ties the oracle to a closed form of the integrator or to
an invariant, not to itself.  No GPU is used here."""
import numpy as np
import pytest

import oracle
import synth


def _lj_state(n, rho, gd, seed, thermostat, kT=1.0, xi=1.0):
    pos, box = synth.lj_box(n, rho, seed)
    vel = synth.mb_velocities(n, kT, seed)
    vel[:, 0] += gd * (pos[:, 2] - 0.5 * box)
    p = oracle.params(box, gd, 2.5, xi=xi, kT=kT, thermostat=thermostat, seed=7, nbins=10)
    return oracle.State(p, pos, vel), box


def test_absolute_and_peculiar_friction_coincide_without_shear():
    """With no shear the streaming velocity is zero everywhere, so the two
    thermostats apply the same force: identical trajectories, bit for bit."""
    a, _ = _lj_state(500, 0.8442, 0.0, 3, thermostat=1)
    b, _ = _lj_state(500, 0.8442, 0.0, 3, thermostat=2)
    assert a.run(40) == oracle.OK and b.run(40) == oracle.OK
    assert np.array_equal(a.pos, b.pos) and np.array_equal(a.vel, b.vel)


@pytest.mark.parametrize("thermostat", [1, 2])
def test_noise_free_friction_decays_by_the_verlet_factor(thermostat):
    """One particle, no neighbours, kT = 0 (no noise), dv/dt = -xi (v - v_ref)
    with v_ref = v_s(z) e_x for the peculiar friction and 0 for the absolute
    one.  Velocity Verlet with the friction on the half-step velocity maps
    h -> (1 - xi dt) h each step, and v = (1 - xi dt / 2) h, so from the
    second step on v - v_ref shrinks by exactly (1 - xi dt) per step.  z does
    not move (vz = 0), so v_ref stays fixed; x may wrap without effect."""
    box, gd, xi, dt = 12.0, 0.5, 2.0, 0.01
    z = 0.8 * box
    p = oracle.params(box, gd, 2.5, xi=xi, kT=0.0, dt=dt, thermostat=thermostat, nbins=4)
    s = oracle.State(p, [[1.0, 2.0, z]], [[0.7, -0.4, 0.0]])
    assert s.run(1) == oracle.OK
    vref = np.array([gd * (z - 0.5 * box) if thermostat == 1 else 0.0, 0.0, 0.0])
    u1 = s.vel[0] - vref
    k = 25
    assert s.run(k) == oracle.OK
    assert s.pos[0, 2] == z
    np.testing.assert_allclose(s.vel[0] - vref, u1 * (1.0 - xi * dt) ** k, rtol=1e-12, atol=1e-15)
    # the other reference would not have decayed that way (the test tells
    # the two frictions apart): only vx differs between them
    other = np.array([0.0 if thermostat == 1 else gd * (z - 0.5 * box), 0.0, 0.0])
    assert abs((s.vel[0] - other)[0] - (u1 + vref - other)[0] * (1.0 - xi * dt) ** k) > 1e-3


def test_absolute_friction_drags_the_flow_toward_rest():
    """Under shear the absolute friction pulls every particle toward zero lab
    velocity, the peculiar one toward the streaming profile: after a short
    run the mean vx in the top layer is far smaller with xi_abs (the layering
    tendency of Fig. 3), while the peculiar run keeps it near v_s there."""
    gd, xi = 0.5, 5.0
    a, box = _lj_state(2000, 0.8442, gd, 5, thermostat=1, xi=xi)
    b, _ = _lj_state(2000, 0.8442, gd, 5, thermostat=2, xi=xi)
    assert a.run(200, sample_every=1) == oracle.OK
    assert b.run(200, sample_every=1) == oracle.OK
    top_vs = gd * (0.95 * box - 0.5 * box)
    assert a.profile[-1] > 0.6 * top_vs
    assert abs(b.profile[-1]) < 0.35 * top_vs


def test_profiles_count_every_particle_and_hold_equipartition():
    """Density: the bins hold every particle at every sample, so the
    density profile integrates to N.  T_y: with no shear, Langevin at kT = 1
    gives m <vy^2> = kT in every layer (equipartition), to sampling error."""
    n, kT = 2000, 1.0
    # strong friction: the melting lattice re-heats within a few hundred steps
    s, box = _lj_state(n, 0.8442, 0.0, 9, thermostat=1, kT=kT, xi=5.0)
    assert s.run(400) == oracle.OK           # equilibrate
    s.vx_sum[:] = 0.0
    s.vy2_sum[:] = 0.0
    s.count[:] = 0
    nsamp = 300
    assert s.run(nsamp, sample_every=1) == oracle.OK
    assert int(s.count.sum()) == n * nsamp
    rho = s.density_profile(nsamp)
    vbin = box ** 3 / rho.shape[0]
    assert np.isclose((rho * vbin).sum(), n, rtol=0, atol=1e-9)
    ty = s.ty_profile
    assert np.all(np.abs(ty - kT) < 0.08), ty
    assert abs(np.average(ty, weights=s.count) - kT) < 0.03
