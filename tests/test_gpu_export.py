"""le_positions into pinned host arrays (the output exported in pieces of
caller ids, each copied back while the next is exported) equals the one-piece
path into ordinary host memory, bit for bit, in both precisions."""
import numpy as np
import pytest

import synth

le = pytest.importorskip("paper_2109_11083_gb300")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [0, 1])
def test_pinned_export_equals_pageable_export(prec):
    n = 3001                            # pieces of unequal size
    pos, box = synth.lj_box(n, 0.8442, 9)
    vel = synth.mb_velocities(n, 1.0, 9)
    gd = 0.7
    vel[:, 0] += gd * (pos[:, 2] - 0.5 * box)
    sim = le.Sim(box, gd, 2.5, 0.3, seed=9, precision=prec)
    sim.set_particles(pos, vel)
    sim.step(120)                       # several list builds: the rank table is rebuilt
    r1, v1 = sim.positions()
    p2 = torch.empty((n, 3), dtype=torch.float64).pin_memory().numpy()
    v2 = torch.empty((n, 3), dtype=torch.float64).pin_memory().numpy()
    le.le_positions(sim.h, n, p2, v2)
    assert np.array_equal(r1, p2) and np.array_equal(v1, v2)
    sim.close()
