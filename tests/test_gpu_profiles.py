"""GPU parity for the comparison thermostat and the z-profiles of Sec. 3.1:
the Langevin friction on the absolute velocity (the paper's xi_abs runs of
Sec. 2.2 / Fig. 3) and the T_y and density profiles, through the C ABI
against the FP64 oracle on the same seeded inputs.

Tolerances as in the other parity tests: positions within 1e-4 after the
run (FP64), profile counts exact, means within 1e-5 (per-particle
contributions are summed in 2^-20 fixed point)."""
import numpy as np
import pytest

import oracle
import synth
from helpers import le_delta

le = pytest.importorskip("paper_2109_11083_gb300")

pytestmark = pytest.mark.gpu


def _pair(n, gd, seed, thermostat, prec=0, xi=1.0, nbins=10):
    pos, box = synth.lj_box(n, 0.8442, seed)
    vel = synth.mb_velocities(n, 1.0, seed)
    vel[:, 0] += gd * (pos[:, 2] - 0.5 * box)
    sim = le.Sim(box, gd, 2.5, 0.3, seed=4, precision=prec, xi=xi, thermostat=thermostat,
                 profile_bins=nbins, sample_every=1)
    sim.set_particles(pos, vel)
    p = oracle.params(box, gd, 2.5, xi=xi, thermostat=thermostat, seed=4, nbins=nbins)
    return sim, oracle.State(p, pos, vel), p, box


def test_absolute_friction_trajectory_matches_oracle():
    gd = 0.5
    sim, ora, p, box = _pair(2048, gd, 31, thermostat=le.LE_THERMO_ABSOLUTE)
    sim.step(60)
    assert ora.run(60) == oracle.OK
    r, v = sim.positions()
    d = le_delta(r, ora.pos, box, oracle.dX(p, 60))
    assert np.abs(d).max() <= 1e-4
    assert np.abs(v - ora.vel).max() <= 1e-6
    sim.close()


@pytest.mark.parametrize("thermostat", [1, 2])
def test_profiles_match_oracle(thermostat):
    """vx, T_y and density per z bin over 150 sampled steps under shear."""
    gd = 0.5
    sim, ora, p, box = _pair(2048, gd, 33, thermostat=thermostat)
    sim.step(150)
    assert ora.run(150, sample_every=1) == oracle.OK
    vx, ty, rho, cnt = sim.profiles()
    assert np.array_equal(cnt, ora.count)
    assert np.abs(vx - ora.profile).max() <= 1e-5
    assert np.abs(ty - ora.ty_profile).max() <= 1e-5
    np.testing.assert_allclose(rho, ora.density_profile(150), rtol=1e-12)
    vx2, cnt2 = sim.velocity_profile()
    assert np.array_equal(vx2, vx) and np.array_equal(cnt2, cnt)
    sim.close()


def test_absolute_friction_in_fp32_drags_the_flow():
    """FP32 mode: the same qualitative contrast as the oracle pin: under
    strong absolute friction the top layer's mean vx falls far below v_s,
    while the peculiar friction keeps it near the streaming profile."""
    gd, xi = 0.5, 5.0
    out = {}
    for th in (le.LE_THERMO_PECULIAR, le.LE_THERMO_ABSOLUTE):
        sim, _, _, box = _pair(4000, gd, 35, thermostat=th, prec=1, xi=xi)
        sim.step(200)
        vx, ty, rho, cnt = sim.profiles()
        assert np.all(np.isfinite(ty)) and cnt.sum() == 4000 * 200
        out[th] = vx[-1]
        sim.close()
    top_vs = gd * (0.95 * box - 0.5 * box)
    assert out[le.LE_THERMO_PECULIAR] > 0.6 * top_vs
    assert abs(out[le.LE_THERMO_ABSOLUTE]) < 0.35 * top_vs
