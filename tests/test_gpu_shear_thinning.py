"""Shear thinning of a Kremer-Grest melt (chains with WCA, FENE and the
Eq. 12 bending term, Sec. 2.4 parameters) over a shear-rate sweep, the
qualitative result of the paper's viscosity sweep (Sec. 3.2): the Eq. 14
viscosity eta = <sigma_xz> / shear_rate falls as the rate grows past the
chains' relaxation rate.  The paper prints no values (its curves are
figures), so the check is the ordering of eta across rates, each with a
block-averaged error, plus the steady-state energy balance that ties the
stress to the temperature: the shear work <sigma_xz> shear_rate V equals
what the Langevin thermostat removes, 3 N xi (T_pec - kT).  (At the highest
rate that balance sets T_pec near 3: viscous heating.)  The rates run
together as one batch, FP32 forces.  The melt is prepared at rest with
dt = 0.01; under shear the step is dt = 0.005, since at T_pec ~ 3 the
0.01 step lets a fast WCA collision throw a bead past the FENE limit R0
(a broken bond) once in a while."""
import numpy as np
import pytest

import synth

le = pytest.importorskip("paper_2109_11083_gb300")

pytestmark = pytest.mark.gpu

RC = 2 ** (1 / 6)
RATES = (0.01, 0.1, 1.0)
XI = 0.5


def _melt(gd, pos, vel, box, bonds, seed, dt=0.01):
    sim = le.Sim(box, gd, RC, 0.3, dt=dt, xi=XI, seed=seed, system_id=seed,
                 precision=1, angle_k=1.5, sample_every=1)
    sim.set_bonds(bonds)
    sim.set_particles(pos, vel)
    return sim


def _sums(s):
    _, avg, n = s.stress(instantaneous=False)
    return avg * n, s.temperature() * n, n


def _block_means(sims, batch, blocks, steps):
    """Mean sigma_xz and T_pec of each block of steps, from the running sums."""
    prev = [_sums(s) for s in sims]
    sxz = np.zeros((len(sims), blocks))
    tpe = np.zeros((len(sims), blocks))
    for k in range(blocks):
        batch.step(steps)
        for m, s in enumerate(sims):
            cur = _sums(s)
            dn = cur[2] - prev[m][2]
            sxz[m, k] = (cur[0] - prev[m][0]) / dn
            tpe[m, k] = (cur[1] - prev[m][1]) / dn
            prev[m] = cur
    return sxz, tpe


def _mean_err(x):
    return x.mean(axis=1), x.std(axis=1, ddof=1) / np.sqrt(x.shape[1])


def test_kremer_grest_melt_thins_under_shear():
    pos, box, bonds = synth.lattice_chains(135, 25, 0.85, 23)
    n = pos.shape[0]
    vel = synth.mb_velocities(n, 1.0, 23)
    eq = _melt(0.0, pos, vel, box, bonds, 23)
    eq.step(20000)  # melt the lattice at rest
    pos, vel = eq.positions()
    eq.close()
    sims = []
    for m, gd in enumerate(RATES):
        v = vel.copy()
        v[:, 0] += gd * (pos[:, 2] - 0.5 * box)
        sims.append(_melt(gd, pos, v, box, bonds, 100 + m, dt=0.005))
    with le.Batch() as b:
        for s in sims:
            b.add(s)
        b.step(20000)  # start-up transient (100 time units)
        sxz, tpe = _block_means(sims, b, 8, 10000)
    for s in sims:
        s.close()
    rates = np.array(RATES)
    s_mean, s_err = _mean_err(sxz)
    t_mean, t_err = _mean_err(tpe)
    eta, err = s_mean / rates, s_err / rates
    print("shear rate, eta, error, T_pec:",
          [(g, round(float(e), 3), round(float(d), 3), round(float(t), 3))
           for g, e, d, t in zip(RATES, eta, err, t_mean)])
    assert np.all(eta > 0)
    # thinning: each tenfold rise of the rate lowers eta beyond the errors
    assert eta[2] < eta[1] - 3 * np.hypot(err[1], err[2])
    assert eta[2] < 0.75 * eta[1]
    assert eta[1] < eta[0] + 3 * np.hypot(err[0], err[1])
    # energy balance: shear work in = thermostat heat out (per unit time)
    V = float(box) ** 3
    work = s_mean * rates * V
    heat = 3 * n * XI * (t_mean - 1.0)
    assert abs(heat[2] - work[2]) < 0.1 * work[2], (heat, work)
    assert abs(heat[1] - work[1]) < 0.3 * work[1] + 3 * 3 * n * XI * t_err[1], (heat, work)
    assert abs(t_mean[0] - 1.0) < 0.02
