"""Long runs against the FP64 oracle (through the C ABI).

1. Steady shear, statistically (Sec. 3.1 profiles; Eqs. 14-15): an LJ fluid
   (N = 1372, rho = 0.8442, shear rate 0.5, Langevin xi = 1 on peculiar
   velocities, kT = 1, dt = 0.005) run for 12,500 steps by the oracle and,
   independently, by the GPU in FP64 and in FP32.  Over the last 20% of the
   steps (the paper's averaging window), in 10 blocks of 250 sampled steps:
   the slope of the vx(z) profile (least squares over 10 bins) must agree
   with the oracle's within 2%, and the viscosity eta = <sigma_xz> / shear
   rate within three combined block standard errors.  The trajectories share
   seeds and start state but decorrelate within a few hundred steps, so the
   comparison is of steady-state averages, not of paths.
2. The plain FP64 LJ-fluid workload as stated (fcc 4000, rho 0.8442, shear
   rate 0.1, xi = 1, dt = 0.005, 500 steps): forces at every one of the 500
   steps within relative 1e-5, final positions within 1e-4, the Eq. 15 xz
   stress (instantaneous and the 500-step running mean) and the 20-bin vx
   profile against the oracle.
"""
import threading

import numpy as np
import pytest

import oracle
import synth
from helpers import force_errors, le_delta

le = pytest.importorskip("paper_2109_11083_gb300")

pytestmark = pytest.mark.gpu

N_LONG, RHO, GD, DT, XI = 1372, 0.8442, 0.5, 0.005, 1.0
STEPS, BLOCKS, NBINS = 12500, 10, 10
WINDOW = STEPS // 5
BLOCK = WINDOW // BLOCKS


def _start():
    pos, box = synth.lj_box(N_LONG, RHO, 77)
    vel = synth.mb_velocities(N_LONG, 1.0, 77)
    vel[:, 0] += GD * (pos[:, 2] - 0.5 * box)
    return pos, vel, box


def _slope(vx_mean, box):
    z = (np.arange(NBINS) + 0.5) * box / NBINS
    return float(np.polyfit(z, vx_mean, 1)[0])


def _oracle_run(out):
    pos, vel, box = _start()
    p = oracle.params(box, GD, 2.5, dt=DT, xi=XI, kT=1.0, seed=5, nbins=NBINS)
    st = oracle.State(p, pos, vel)
    assert st.run(STEPS - WINDOW) == oracle.OK
    blocks = []
    prev = 0.0
    for _ in range(BLOCKS):
        assert st.run(BLOCK, sample_every=1) == oracle.OK
        blocks.append((st.samples.sxz_sum - prev) / BLOCK)
        prev = st.samples.sxz_sum
    out["eta_blocks"] = np.array(blocks) / GD
    out["profile"] = st.profile.copy()
    out["box"] = box


def _gpu_run(prec):
    pos, vel, box = _start()
    sim = le.Sim(box, GD, 2.5, 0.3, dt=DT, xi=XI, kT=1.0, seed=5, precision=prec,
                 profile_bins=NBINS, sample_every=1)
    sim.set_particles(pos, vel)
    sim.step(STEPS - WINDOW)
    eta, vx_sum, cnt_sum = [], np.zeros(NBINS), np.zeros(NBINS)
    for _ in range(BLOCKS):
        sim.reset_samples()
        sim.step(BLOCK)
        _, xz, ns = sim.stress(instantaneous=False)
        assert ns == BLOCK
        eta.append(xz / GD)
        vx, cnt = sim.velocity_profile()
        vx_sum += np.nan_to_num(vx) * cnt
        cnt_sum += cnt
    sim.close()
    return np.array(eta), vx_sum / cnt_sum, box


def _stats(blocks):
    return float(blocks.mean()), float(blocks.std(ddof=1) / np.sqrt(blocks.size))


def test_steady_shear_profile_slope_and_viscosity_match_oracle():
    ora = {}
    th = threading.Thread(target=_oracle_run, args=(ora,))   # the oracle's C code runs
    th.start()                                               # without the GIL
    gpu = {prec: _gpu_run(prec) for prec in (0, 1)}
    th.join()
    eta_o, err_o = _stats(ora["eta_blocks"])
    slope_o = _slope(ora["profile"], ora["box"])
    assert eta_o > 0 and abs(slope_o / GD - 1.0) < 0.05
    for prec, (eta_blocks, prof, box) in gpu.items():
        eta_g, err_g = _stats(eta_blocks)
        slope_g = _slope(prof, box)
        comb = np.hypot(err_o, err_g)
        print(f"\nprec={prec}: slope {slope_g:.5f} vs oracle {slope_o:.5f} "
              f"({abs(slope_g / slope_o - 1):.2%}); eta {eta_g:.4f} +- {err_g:.4f} vs oracle "
              f"{eta_o:.4f} +- {err_o:.4f} (difference {abs(eta_g - eta_o) / comb:.2f} combined "
              f"errors, {abs(eta_g / eta_o - 1):.2%})")
        assert abs(slope_g / slope_o - 1.0) <= 0.02
        assert abs(eta_g - eta_o) <= 3.0 * comb


def test_lj_fluid_4000_fp64_500_steps_as_stated():
    w = synth.lj_fluid_4000()
    assert w.n == 4000 and w.steps == 500 and w.precision == 0
    pos, vel = synth.lj_initial_state(w)
    vel[:, 0] += w.shear_rate * (pos[:, 2] - 0.5 * w.box)
    sim = le.Sim(w.box, w.shear_rate, w.rc, w.skin, dt=w.dt, xi=w.xi, kT=w.kT, seed=w.seed,
                 precision=0, profile_bins=20, sample_every=1)
    sim.set_particles(pos, vel)
    p = oracle.params(w.box, w.shear_rate, w.rc, dt=w.dt, xi=w.xi, kT=w.kT, seed=w.seed,
                      nbins=20)
    ora = oracle.State(p, pos, vel)
    worst = (0.0, 0.0)
    for step in range(1, w.steps + 1):
        sim.step(1)
        assert ora.run(1, sample_every=1) == oracle.OK
        g, q = force_errors(sim.forces(), ora.Fc)
        assert g <= 1e-5 and q <= 1e-5, (step, g, q)
        worst = (max(worst[0], g), max(worst[1], q))
    r, v = sim.positions()
    dpos = np.abs(le_delta(r, ora.pos, w.box, oracle.dX(p, w.steps))).max()
    assert dpos <= 1e-4
    S, xz, ns = sim.stress()
    S_ref, _, _ = ora.observe()
    assert ns == w.steps == ora.samples.nsamples
    assert abs(S[0, 2] - S_ref[0, 2]) <= 1e-8 * np.abs(S_ref).max()
    xz_ref = ora.samples.sxz_sum / w.steps
    assert xz == pytest.approx(xz_ref, rel=1e-7, abs=1e-9)
    vx, cnt = sim.velocity_profile()
    assert np.array_equal(cnt, ora.count)
    assert np.abs(vx - ora.profile).max() <= 1e-5
    print(f"\nfcc 4000, 500 FP64 steps: worst force errors {worst}, positions {dpos:.2e}, "
          f"<sigma_xz> {xz:.6f} vs {xz_ref:.6f}")
    sim.close()
