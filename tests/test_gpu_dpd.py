"""GPU parity for the DPD thermostat (Eqs. 6-8, the pairwise friction and
noise along the bond with weight w = 1 - r/rc, the image's velocity shifted
by the shear across the sheared faces): through the C ABI against the FP64
oracle on the same seeded inputs.  FP64: the trajectory within the tolerances
of the Langevin parity tests; momentum conserved without shear; FP32: the
temperature held at kT."""
import numpy as np
import pytest

import oracle
import synth
from helpers import le_delta

le = pytest.importorskip("paper_2109_11083_gb300")

pytestmark = pytest.mark.gpu


def _pair(n, gd, seed, prec=0, xi=4.5, nbins=10):
    pos, box = synth.lj_box(n, 0.8442, seed)
    vel = synth.mb_velocities(n, 1.0, seed)
    vel[:, 0] += gd * (pos[:, 2] - 0.5 * box)
    sim = le.Sim(box, gd, 2.5, 0.3, seed=4, system_id=9, precision=prec, xi=xi,
                 thermostat=le.LE_THERMO_DPD, profile_bins=nbins, sample_every=1)
    sim.set_particles(pos, vel)
    p = oracle.params(box, gd, 2.5, xi=xi, thermostat=3, seed=4, system=9, nbins=nbins)
    return sim, oracle.State(p, pos, vel), p, box


@pytest.mark.parametrize("gd", [0.0, 0.5])
def test_dpd_trajectory_matches_oracle(gd):
    sim, ora, p, box = _pair(2048, gd, 41)
    for k in (1, 20, 60):
        sim.step(k - sim.counters()["step"])
        assert ora.run(k - ora.step.value) == oracle.OK
        r, v = sim.positions()
        d = le_delta(r, ora.pos, box, oracle.dX(p, k))
        assert np.abs(d).max() <= 1e-4, (k, np.abs(d).max())
        assert np.abs(v - ora.vel).max() <= 1e-6, (k, np.abs(v - ora.vel).max())
    if gd > 0:
        assert sim.counters()["rebuilds"] > 0
    sim.close()


def test_dpd_profiles_and_stress_match_oracle():
    sim, ora, p, box = _pair(2048, 0.5, 43)
    sim.step(80)
    assert ora.run(80, sample_every=1) == oracle.OK
    vx, ty, rho, cnt = sim.profiles()
    assert np.array_equal(cnt, ora.count)
    assert np.abs(vx - ora.profile).max() <= 1e-5
    assert np.abs(ty - ora.ty_profile).max() <= 1e-5
    S, _, _ = sim.stress()
    S_ref, _, _ = ora.observe()
    assert np.abs(S - S_ref).max() <= 1e-6 * np.abs(S_ref).max()
    sim.close()


def test_dpd_conserves_momentum_without_shear():
    """Every DPD pair force is applied with both signs from one shared
    random number, so the total momentum stays where it started."""
    sim, _, _, _ = _pair(3000, 0.0, 45)
    _, v0 = sim.positions()
    P0 = v0.sum(axis=0)
    sim.step(200)
    _, v = sim.positions()
    assert np.abs(v.sum(axis=0) - P0).max() < 1e-9 * 3000
    sim.close()


def test_dpd_fp32_holds_the_temperature():
    sim, _, _, _ = _pair(8000, 0.0, 47, prec=1)
    sim.step(300)
    T = []
    for _ in range(10):
        sim.step(20)
        _, v = sim.positions()
        v = v - v.mean(axis=0)
        T.append((v * v).sum() / (3 * v.shape[0] - 3))
    assert abs(np.mean(T) - 1.0) < 0.04, T
    sim.close()
