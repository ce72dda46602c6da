"""GPU parity: the CUDA path (called through the C ABI) against the FP64 CPU
oracle on the same seeded inputs.

Tolerances.  Both precisions: per-step forces within a relative 1e-5 (global
L2 over all components, and per particle against max(|F_i|, <|F|>)) and
10-step positions within 1e-4.  In FP32 mode a pair whose distance lies within
the rounding band of the strict cut-off (|r - rc| <= 4 sqrt(3) u (6P + 2 rc),
u = 2^-24, P the largest reference-relative coordinate) may be counted or not:
either is a correct FP32 result, so the comparison takes the FP32 path's
decision for those pairs (oracle.band_pairs) and reports how many it took the
other way instead of counting them as error.  Each particle's FP32 force error
must in addition lie within the first-order rounding bound B_i that the oracle
derives from the arithmetic (oracle.force_error_bound: separation error
u(6P + 2r) per component times the norm of dF/dd, plus evaluation and
summation rounding, plus the whole pair force of band pairs), and the L2 error
over all particles within the L2 norm of B.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from helpers import flip_resolved_errors, force_errors, le_delta

le = pytest.importorskip("paper_2109_11083_gb300")

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-5
FP64_FORCE_TOL = FORCE_TOL
POS_TOL = 1e-4
U32 = 2.0 ** -24
# worst FP32 errors seen by the tests of this module (flip-resolved), printed
# at the end of each FP32 test
FP32_SEEN = {"l2": 0.0, "particle": 0.0, "flips": 0, "band": 0}


@pytest.fixture(autouse=True)
def _fp32_error_report(request):
    """Prints each test's worst FP32 force errors (flip-resolved), the
    measured statement of the FP32 path's force error."""
    for k in FP32_SEEN:
        FP32_SEEN[k] = 0 if k in ("flips", "band") else 0.0
    yield
    if FP32_SEEN["l2"] > 0.0:
        print(f"\nFP32 force error [{request.node.name}]: global L2 {FP32_SEEN['l2']:.3e}, "
              f"per particle {FP32_SEEN['particle']:.3e}, band pairs {FP32_SEEN['band']}, "
              f"decided the other way {FP32_SEEN['flips']}")


def band_width(P, rc):
    """Distance from the cut-off within which an FP32 separation may fall on
    either side of the strict r < rc test (four times the first-order
    separation bound, so that no flip escapes the comparison)."""
    return 4.0 * math.sqrt(3.0) * U32 * (6.0 * P + 2.0 * rc)


def lj_inputs(n, rho, gd, seed, kT=1.0, jitter=0.0):
    pos, box = synth.lj_box(n, rho, seed)
    if jitter:
        pos = np.mod(pos + np.random.default_rng(seed).uniform(-jitter, jitter, pos.shape), box)
    vel = synth.mb_velocities(n, kT, seed)
    vel[:, 0] += gd * (pos[:, 2] - 0.5 * box)
    return pos, vel, box


def make_pair(pos, vel, box, gd, rc=2.5, skin=0.3, prec=0, bonds=None, seed=1, xi=1.0, kT=1.0,
              dt=0.005, thermostat=1, fene_k=30.0, nbins=20, sample_every=1):
    sim = le.Sim(box, gd, rc, skin, dt=dt, xi=xi, kT=kT, seed=seed, precision=prec,
                 thermostat=thermostat, fene_k=fene_k, profile_bins=nbins,
                 sample_every=sample_every)
    if bonds is not None:
        sim.set_bonds(bonds)
    sim.set_particles(pos, vel)
    p = oracle.params(box, gd, rc, dt=dt, xi=xi, kT=kT, seed=seed, thermostat=thermostat,
                      fene_k=fene_k if bonds is not None else 0.0, nbins=nbins)
    ora = oracle.State(p, pos, vel, bonds=bonds)
    return sim, ora, p


def ref_extent(box, rc, skin, bonds=None):
    """Largest reference-relative coordinate P: half a cell edge (cells of
    edge >= rc + skin, and >= R0 with bonds) plus half the skin."""
    L = np.broadcast_to(np.asarray(box, dtype=np.float64), (3,))
    edge = max(rc + skin, 1.5 if bonds is not None else 0.0)
    lc = max(L[a] / math.floor(L[a] / edge) for a in range(3))
    return 0.5 * lc + 0.5 * skin


def assert_forces(f, ref, prec, what="", bound=None, band=None, rows=None,
                  particle_tol=FORCE_TOL):
    """FP64: the 1e-5 relative force tolerance directly.  FP32: the same tolerance once
    the band pairs' cut-off decisions are taken out (band = oracle.band_pairs
    output), and every particle within the rounding bound; particle_tol
    replaces the per-particle tolerance where the configuration's forces are
    far smaller than the pair forces they sum (stated per test)."""
    g, q = force_errors(f, ref)
    if prec == 0:
        assert g <= FP64_FORCE_TOL and q <= FP64_FORCE_TOL, (what, g, q)
        return g, q
    err = np.linalg.norm(np.asarray(f) - np.asarray(ref), axis=1)
    worst = int(np.argmax(err / bound))
    assert np.all(err <= bound), (what, worst, err[worst], bound[worst])
    assert np.linalg.norm(err) <= np.linalg.norm(bound), (what, g)
    g, q, flips, nband = flip_resolved_errors(f, ref, *band, rows=rows)
    FP32_SEEN["l2"] = max(FP32_SEEN["l2"], g)
    FP32_SEEN["particle"] = max(FP32_SEEN["particle"], q)
    FP32_SEEN["flips"] += flips
    FP32_SEEN["band"] += nband
    assert g <= FORCE_TOL and q <= particle_tol, (what, g, q, flips)
    return g, q


def check_at_gpu_positions(sim, p, step, prec, box, rc, skin, bonds=None, use_cells=True,
                           particle_tol=FORCE_TOL):
    """Oracle forces (and, in FP32 mode, the rounding bound) at the GPU's own
    positions after `step` steps, against the GPU forces."""
    r, _ = sim.positions()
    dX = oracle.dX(p, step)
    st, F, _, _ = oracle.forces(p, dX, r, bonds, use_cells=use_cells)
    assert st == oracle.OK
    B = band = None
    if prec == 1:
        P = ref_extent(box, rc, skin, bonds)
        B = oracle.force_error_bound(p, dX, r, bonds, U32, P)
        band = oracle.band_pairs(p, dX, r, band_width(P, rc))
    return assert_forces(sim.forces(), F, prec, f"step {step}", B, band,
                         particle_tol=particle_tol)


@pytest.mark.parametrize("prec", [0, 1])
def test_initial_forces_match_oracle(prec):
    pos, vel, box = lj_inputs(4000, 0.8442, 0.1, 3, jitter=0.1)
    sim, ora, p = make_pair(pos, vel, box, 0.1, prec=prec)
    check_at_gpu_positions(sim, p, 0, prec, box, 2.5, 0.3)
    assert np.abs(sim.forces() - ora.Fc).max() <= 1e-3
    sim.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_forces_every_step_at_high_shear_match_oracle_at_gpu_positions(prec):
    """High shear so the image offset sweeps the whole box and the lists are
    rebuilt many times by the image-shift term; at every step the GPU forces
    equal the oracle's forces evaluated at the GPU's own positions."""
    gd = 1.0
    pos, vel, box = lj_inputs(2048, 0.8442, gd, 11)
    sim, _, p = make_pair(pos, vel, box, gd, prec=prec)
    worst = (0.0, 0.0)
    for step in range(1, 241):
        sim.step(1)
        r, _ = sim.positions()
        c = sim.counters()
        assert c["step"] == step
        dX = oracle.dX(p, step)
        assert c["dX"] == dX
        g, q = check_at_gpu_positions(sim, p, step, prec, box, 2.5, 0.3)
        worst = (max(worst[0], g), max(worst[1], q))
    c = sim.counters()
    assert c["rebuilds"] >= 20
    assert dX > 0 and gd * box * 240 * 0.005 > box      # the offset wrapped at least once
    print(f"prec={prec} worst force errors {worst}, rebuilds {c['rebuilds']} "
          f"(image-forced {c['image_rebuilds']})")
    sim.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_cold_sheared_crystal_rebuilds_on_the_shear_term(prec):
    """A cold crystal under strong shear: the peculiar displacements stay tiny,
    so the lists are rebuilt on the shear term of the trigger (the spread of
    streaming displacements across a pair) rather than on the displacements;
    streaming itself and the drift of the image offset do not force builds.
    Forces stay exact throughout.  At kT = 0.02 a particle's force is ~50
    times smaller than the pair forces it sums, so FP32 rounding of the pair
    arithmetic alone (exact separations) reaches ~2e-5 of it: the FP32
    per-particle tolerance here is 5e-5 (the global L2 one stays 1e-5)."""
    gd = 2.0
    pos, vel, box = lj_inputs(2048, 0.8442, gd, 19, kT=0.02)
    sim, _, p = make_pair(pos, vel, box, gd, prec=prec, kT=0.02, xi=10.0)
    for step in range(1, 151):
        sim.step(1)
        if step % 3 == 0:
            check_at_gpu_positions(sim, p, step, prec, box, 2.5, 0.3, particle_tol=5e-5)
    c = sim.counters()
    assert c["image_rebuilds"] >= 2, c
    # far fewer builds than steps although particles stream by up to
    # shear*Lz/2 * dt = 0.07 per step
    assert c["rebuilds"] <= 30, c
    sim.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_trajectory_parity_lj_fluid_4000(prec):
    """The FP64 LJ-fluid workload (fcc 4000, rho 0.8442, shear 0.1, Langevin
    xi = 1 on peculiar velocities): per-step forces and 10-step positions."""
    w = synth.lj_fluid_4000()
    pos, vel = synth.lj_initial_state(w)
    vel[:, 0] += w.shear_rate * (pos[:, 2] - 0.5 * w.box)
    sim, ora, p = make_pair(pos, vel, w.box, w.shear_rate, rc=w.rc, skin=w.skin, prec=prec,
                            seed=w.seed, xi=w.xi, dt=w.dt)
    for step in range(1, 11):
        sim.step(1)
        assert ora.run(1) == oracle.OK
        if prec == 0:
            assert_forces(sim.forces(), ora.Fc, prec, f"step {step}")
        else:
            check_at_gpu_positions(sim, p, step, prec, w.box, w.rc, w.skin)
    r, v = sim.positions()
    d = le_delta(r, ora.pos, w.box, oracle.dX(p, 10))
    assert np.abs(d).max() <= POS_TOL
    assert np.abs(v - ora.vel).max() <= (1e-9 if prec == 0 else 1e-4)
    print(f"\nprec={prec} 10-step position error {np.abs(d).max():.3e}, "
          f"velocity error {np.abs(v - ora.vel).max():.3e}")
    sim.close()


def test_observables_match_oracle_fp64():
    """Eq. 15 stress (instantaneous tensor and running xz mean), the vx(z)
    profile and the peculiar temperature over 200 sampled steps."""
    gd = 0.5
    pos, vel, box = lj_inputs(2048, 0.8442, gd, 21)
    sim, ora, p = make_pair(pos, vel, box, gd, nbins=10)
    sim.step(200)
    assert ora.run(200, sample_every=1) == oracle.OK
    S, xz, ns = sim.stress()
    S_ref, t_ref, _ = ora.observe()
    assert ns == 200 == ora.samples.nsamples
    assert np.abs(S - S_ref).max() <= 1e-8 * np.abs(S_ref).max()
    assert xz == pytest.approx(ora.samples.sxz_sum / 200, rel=1e-7, abs=1e-9)
    vx, cnt = sim.velocity_profile()
    assert np.array_equal(cnt, ora.count)
    assert np.abs(vx - ora.profile).max() <= 1e-5
    assert sim.temperature() > 0.5
    sim.close()


def test_observables_fp32_against_oracle():
    """The FP32 path's error in the sampled outputs against the FP64 oracle
    (same seeds, 50 steps, both trajectories start from one state): the Eq. 15
    xz stress (instantaneous and running mean), the vx(z) profile and the
    positions.  The stated FP32 tolerances: relative 1e-4 for the stress,
    1e-4 for the profile means, 1e-4 for positions."""
    gd = 0.5
    pos, vel, box = lj_inputs(2048, 0.8442, gd, 21)
    sim, ora, p = make_pair(pos, vel, box, gd, nbins=10, prec=1)
    sim.step(50)
    assert ora.run(50, sample_every=1) == oracle.OK
    S, xz, ns = sim.stress()
    S_ref, _, _ = ora.observe()
    s_err = abs(S[0, 2] - S_ref[0, 2]) / np.abs(S_ref).max()
    xz_ref = ora.samples.sxz_sum / 50
    xz_err = abs(xz - xz_ref) / abs(xz_ref)
    vx, cnt = sim.velocity_profile()
    prof_err = np.abs(vx - ora.profile).max()
    r, _ = sim.positions()
    pos_err = np.abs(le_delta(r, ora.pos, box, oracle.dX(p, 50))).max()
    print(f"\nFP32 observables after 50 steps: sigma_xz {s_err:.3e} (rel. to max |S|), "
          f"running <sigma_xz> {xz_err:.3e} (rel.), profile {prof_err:.3e} (abs.), "
          f"count differences {int(np.abs(cnt - ora.count).sum())}, positions {pos_err:.3e}")
    assert ns == 50
    assert s_err <= 1e-4 and xz_err <= 1e-4
    assert prof_err <= 1e-4
    assert pos_err <= POS_TOL
    sim.close()


def test_checkpoint_restore_is_bitwise():
    gd = 0.3
    pos, vel, box = lj_inputs(3000, 0.8442, gd, 5)
    a = le.Sim(box, gd, 2.5, 0.3, seed=3, precision=1)
    a.set_particles(pos, vel)
    a.step(37)
    blob = a.get_state()
    a.step(41)
    ra, va = a.positions()
    fa = a.forces()
    b = le.Sim(box, gd, 2.5, 0.3, seed=3, precision=1)
    b.set_particles(pos, vel)
    b.set_state(blob)
    b.step(41)
    rb, vb = b.positions()
    assert np.array_equal(ra, rb) and np.array_equal(va, vb)
    assert np.array_equal(fa, b.forces())
    assert a.counters()["step"] == b.counters()["step"] == 78
    a.close()
    b.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_kremer_grest_chains_fene_parity(prec):
    """WCA (Eq. 10 at rc = 2^(1/6)) + FENE (Eq. 11) chains under strong shear:
    forces at every step against the oracle at the GPU's positions."""
    pos, box, bonds = synth.lattice_chains(40, 25, 0.85, 13)
    gd = 0.5
    vel = synth.mb_velocities(pos.shape[0], 1.0, 13)
    vel[:, 0] += gd * (pos[:, 2] - 0.5 * box)
    rc = 2 ** (1 / 6)
    sim, ora, p = make_pair(pos, vel, box, gd, rc=rc, skin=0.3, prec=prec, bonds=bonds,
                            dt=0.005, xi=0.5)
    check_at_gpu_positions(sim, p, 0, prec, box, rc, 0.3, bonds)
    for step in range(1, 201):
        sim.step(1)
        if step % 5 == 0:
            check_at_gpu_positions(sim, p, step, prec, box, rc, 0.3, bonds)
    assert sim.counters()["rebuilds"] > 0
    sim.close()


def test_broken_bond_is_reported_and_rolled_back():
    pos = np.array([[2.0, 2.0, 2.0], [3.0, 2.0, 2.0], [5.0, 5.0, 5.0]])
    vel = np.array([[-30.0, 0, 0], [30.0, 0, 0], [0, 0, 0]])
    sim = le.Sim(10.0, 0.0, 2 ** (1 / 6), 0.3, thermostat=0, dt=0.01)
    sim.set_bonds([[0, 1]])
    sim.set_particles(pos, vel)
    r0, v0 = sim.positions()
    with pytest.raises(le.LEError) as e:
        sim.step(50)
    assert e.value.status == 5
    r1, v1 = sim.positions()
    assert np.array_equal(r0, r1) and np.array_equal(v0, v1)
    assert sim.counters()["step"] == 0
    sim.close()


@pytest.mark.parametrize("n", [1, 2, 33, 257])
def test_tiny_and_ragged_systems(n):
    """Sizes that fill no warp or block evenly; one particle is a free particle
    on the sheared image lattice."""
    gd = 0.7
    box = np.array([9.0, 8.0, 7.5])
    g = np.random.default_rng(n)
    # fcc sites of a cube of the same volume, stretched onto the box, keep
    # every periodic image at least ~1 apart
    cube, L0 = synth.lj_box(n, n / float(np.prod(box)), n)
    pos = cube * (box / L0)
    vel = g.normal(size=(n, 3))
    sim, ora, p = make_pair(pos, vel, box, gd, thermostat=0, prec=0)
    for _ in range(5):
        sim.step(20)
        assert ora.run(20) == oracle.OK
    r, v = sim.positions()
    d = le_delta(r, ora.pos, box, oracle.dX(p, 100))
    assert np.abs(d).max() <= 1e-9
    assert np.abs(v - ora.vel).max() <= 1e-9
    sim.close()


def test_two_cells_per_dimension_small_box():
    """N = 500 at rho = 0.9: L = 8.22 gives only 2 cells of edge >= 2.8, so a
    neighbour cell is reached through two different images."""
    gd = 0.2
    pos, vel, box = lj_inputs(500, 0.9, gd, 17)
    sim, _, p = make_pair(pos, vel, box, gd, prec=1)
    assert sim.counters()["cells"] == (2, 2, 2)
    for step in range(1, 101):
        sim.step(1)
        if step % 10 == 0:
            check_at_gpu_positions(sim, p, step, 1, box, 2.5, 0.3, use_cells=False)
    sim.close()


def test_negative_shear_and_zero_shear():
    for gd in (-0.8, 0.0):
        pos, vel, box = lj_inputs(1372, 0.8442, gd, 31)
        sim, ora, p = make_pair(pos, vel, box, gd, prec=0)
        sim.step(60)
        assert ora.run(60) == oracle.OK
        assert_forces(sim.forces(), ora.Fc, 0, f"shear {gd}")
        sim.close()


def test_full_size_box_sampled_forces():
    """The 4,194,304-particle box in the benchmark's launch configuration:
    after a few steps, forces on 3000 sampled particles against the oracle's
    one-particle-at-a-time sums."""
    w = synth.lj_box_4m()
    pos, vel = synth.lj_initial_state(w)
    vel[:, 0] += w.shear_rate * (pos[:, 2] - 0.5 * w.box)
    sim = le.Sim(w.box, w.shear_rate, w.rc, w.skin, dt=w.dt, xi=w.xi, seed=w.seed, precision=1)
    sim.set_particles(pos, vel)
    sim.step(12)
    r, _ = sim.positions()
    f = sim.forces()
    p = oracle.params(w.box, w.shear_rate, w.rc)
    idx = np.random.default_rng(0).choice(w.n, 3000, replace=False)
    dX = oracle.dX(p, 12)
    F = oracle.forces_on(p, dX, r, idx)
    # the rounding bound needs every pair of the sampled particles: take it
    # from the sampled particles' neighbourhood (a sub-box around each would
    # do; the full box is used once, with the cell list)
    P = ref_extent(w.box, w.rc, w.skin)
    B = oracle.force_error_bound(p, dX, r, None, U32, P)[idx]
    band = oracle.band_pairs(p, dX, r, band_width(P, w.rc))
    assert_forces(f[idx], F, 1, "full size", B, band, rows=idx)
    assert sim.counters()["rebuilds"] >= 1
    sim.close()


def test_profile_value_out_of_range_is_reported_and_rolled_back():
    """A sampled |vx| above the fixed-point range of the profile sums (1000)
    is an error with the state rolled back, not a silently clamped sum."""
    pos = np.array([[2.0, 2.0, 2.0], [6.0, 6.0, 6.0]])
    vel = np.array([[1500.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    sim = le.Sim(10.0, 0.0, 2.5, 0.3, thermostat=0, dt=0.0001, profile_bins=4)
    sim.set_particles(pos, vel)
    r0, v0 = sim.positions()
    with pytest.raises(le.LEError) as e:
        sim.step(3)
    assert e.value.status == 10
    r1, v1 = sim.positions()
    assert np.array_equal(r0, r1) and np.array_equal(v0, v1)
    assert sim.counters()["step"] == 0
    sim.close()
    # within range the same system steps and samples normally
    vel[0, 0] = 900.0
    sim = le.Sim(10.0, 0.0, 2.5, 0.3, thermostat=0, dt=0.0001, profile_bins=4)
    sim.set_particles(pos, vel)
    sim.step(3)
    vx, cnt = sim.velocity_profile()
    assert cnt.sum() == 6 and np.nanmax(vx) == pytest.approx(900.0, rel=1e-6)
    sim.close()


def test_set_particles_again_equals_a_fresh_handle():
    """A second le_set_particles with the same layout reuses the device
    buffers and step graphs: the run from it equals the same run on a fresh
    handle bit for bit; a non-finite input fails the call (the import kernel
    finds it) and leaves the handle usable."""
    gd = 0.4
    pos1, vel1, box = lj_inputs(2000, 0.8442, gd, 41)
    pos2, vel2, _ = lj_inputs(2000, 0.8442, gd, 43)
    a = le.Sim(box, gd, 2.5, 0.3, seed=9, precision=1)
    a.set_particles(pos1, vel1)
    a.step(25)
    bad = pos2.copy()
    bad[17, 1] = np.nan
    with pytest.raises(le.LEError) as e:
        a.set_particles(bad, vel2)
    assert e.value.status == 1
    a.set_particles(pos2, vel2)
    a.step(40)
    b = le.Sim(box, gd, 2.5, 0.3, seed=9, precision=1)
    b.set_particles(pos2, vel2)
    b.step(40)
    ra, va = a.positions()
    rb, vb = b.positions()
    assert np.array_equal(ra, rb) and np.array_equal(va, vb)
    assert np.array_equal(a.forces(), b.forces())
    a.close()
    b.close()
