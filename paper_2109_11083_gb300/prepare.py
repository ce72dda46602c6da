"""Initial conditions that need the library itself: the push-off of
overlapping random-walk chains.

Freely jointed random walks (bond 0.97, the Kremer-Grest melt of the paper's
Sec. 2.4) overlap; integrated as they are, the WCA force between overlapping
beads is far too large for any time step.  The push-off runs Langevin
dynamics at rest with every LJ pair force limited to a cap (le_params
force_cap, FP64), raising the cap stage by stage until it exceeds the forces
of a dense melt, so that the chains relax apart; the melt is then equilibrated
without a cap by the caller.
"""
from __future__ import annotations

import numpy as np

from . import LE_FP64, Sim

# the cap of each stage (reduced LJ force units) and the steps per stage
PUSH_OFF_CAPS = (10.0, 30.0, 100.0, 300.0, 1000.0)
PUSH_OFF_STEPS = 400


def push_off(pos, box, bonds, *, caps=PUSH_OFF_CAPS, steps_per_cap=PUSH_OFF_STEPS,
             rc=2 ** (1 / 6), skin=0.3, dt=0.005, xi=1.0, kT=1.0, fene_k=30.0, fene_R0=1.5,
             seed=0, stream=None):
    """Positions and velocities of the chains after the capped push-off (no
    shear, peculiar Langevin thermostat, WCA + FENE).  Velocities start at
    zero; the thermostat brings them to kT."""
    pos = np.array(pos, dtype=np.float64)
    vel = np.zeros_like(pos)
    for k, cap in enumerate(caps):
        sim = Sim(box, 0.0, rc, skin, stream=stream, dt=dt, xi=xi, kT=kT, seed=seed + k,
                  precision=LE_FP64, fene_k=fene_k, fene_R0=fene_R0, force_cap=float(cap),
                  sample_every=0)
        sim.set_bonds(bonds)
        sim.set_particles(pos, vel)
        sim.step(steps_per_cap)
        pos, vel = sim.positions()
        sim.close()
    return pos, vel
