"""The allocation-free force entry point, le_forces_noalloc, for callers that
cannot allocate device memory where they need forces: its output must equal
the forces a handle computes for the same positions and step (le_forces),
and the FP64 oracle's forces, within the tolerances of the other GPU tests
(relative 1e-5; in FP32 once the cut-off decisions of pairs within the
rounding band of rc are taken out), on two calls in a row (the second reuses
the static device array the first one left behind).

Collected last on purpose (file name), so a run that stops at the first
failure has already run every other test."""
import math

import numpy as np
import pytest

import oracle
import synth
from helpers import flip_resolved_errors, force_errors

le = pytest.importorskip("paper_2109_11083_gb300")

pytestmark = pytest.mark.gpu


def _system(n, rho, gd, seed):
    pos, box = synth.lj_box(n, rho, seed)
    vel = synth.mb_velocities(n, 1.0, seed)
    vel[:, 0] += gd * (pos[:, 2] - 0.5 * box)
    return pos, vel, box


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_forces_equal_handle_forces_twice(prec):
    gd, rc, skin = 0.7, 2.5, 0.3
    pos, vel, box = _system(6000, 0.8442, gd, 41 + prec)
    sim = le.Sim(box, gd, rc, skin, seed=2, precision=prec)
    sim.set_particles(pos, vel)
    params = le.le_default_params()
    params.precision = prec
    for call in range(2):
        sim.step(37)                              # a non-zero image offset
        step = sim.counters()["step"]
        r, _ = sim.positions()
        f_ref = sim.forces()
        f = le.le_forces_noalloc(box, gd, rc, skin, params, step, r)
        p = oracle.params(box, gd, rc)
        dX = oracle.dX(p, step)
        st, F, _, _ = oracle.forces(p, dX, r)
        assert st == oracle.OK
        if prec == 0:
            g, q = force_errors(f, f_ref)
            assert g <= 1e-5 and q <= 1e-5, (call, g, q)
            g, q = force_errors(f, F)
            assert g <= 1e-5 and q <= 1e-5, (call, g, q)
        else:
            # against the oracle: the 1e-5 relative force tolerance once the band
            # pairs' cut-off decisions are taken out
            P = 0.5 * box / math.floor(box / (rc + skin))
            band = 4.0 * math.sqrt(3.0) * 2.0 ** -24 * (6.0 * P + 2.0 * rc)
            g, q, flips, _ = flip_resolved_errors(f, F, *oracle.band_pairs(p, dX, r, band))
            assert g <= 1e-5 and q <= 1e-5, (call, g, q, flips)
            # both sides round positions to FP32 around different cell
            # references: each may differ from the exact forces by the
            # oracle's rounding bound, so together by twice that
            edge = rc + skin
            P = 0.5 * box / math.floor(box / edge) + 0.5 * skin
            B = oracle.force_error_bound(p, oracle.dX(p, step), r, None, 2.0 ** -24, P)
            err = np.linalg.norm(f - f_ref, axis=1)
            assert np.all(err <= 2 * B), call
    sim.close()


def test_noalloc_rejects_sizes_beyond_its_static_array():
    pos, _, box = _system(20000, 0.8442, 0.1, 5)
    with pytest.raises(le.LEError) as e:
        le.le_forces_noalloc(box, 0.1, 2.5, 0.3, le.le_default_params(), 0, pos)
    assert e.value.status == 1
