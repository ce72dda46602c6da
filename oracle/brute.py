"""TEST INFRASTRUCTURE ONLY: image-enumeration force sum in numpy.

The plain definition of the forces under sheared periodic images (Fig. 1,
Eq. 4): the image of particle j in box (nx, ny, nz) sits at
    r_j + (nx*Lx + nz*dX, ny*Ly, nz*Lz),
and particle i feels every image of every particle (itself included, apart
from its own zero image) that lies within rc.  No minimum-image convention is
used, so this pins the oracle's minimum-image code from the outside.
Only for tiny systems (O(N^2 * images)).
"""
from __future__ import annotations

import itertools

import numpy as np


def lj_f_over_r(r2, eps=1.0, sigma=1.0):
    """Eq. 9: -dV/dr / r for V = 4 eps [(s/r)^12 - (s/r)^6]."""
    s6 = (sigma * sigma / r2) ** 3
    return 24.0 * eps * (2.0 * s6 * s6 - s6) / r2


def lj_energy(r2, eps=1.0, sigma=1.0, rc=None):
    """Eq. 9, shifted by its value at rc as in Eq. 10 when rc is given."""
    s6 = (sigma * sigma / r2) ** 3
    e = 4.0 * eps * (s6 * s6 - s6)
    if rc is not None:
        c6 = (sigma / rc) ** 6
        e -= 4.0 * eps * (c6 * c6 - c6)
    return e


def image_forces(pos, box, dX, rc, eps=1.0, sigma=1.0, reach=2):
    """Forces, virial sum_{i<j} r_ij (x) F_ij and the number of interacting
    (i, image-of-j) pairs, by explicit enumeration of image boxes."""
    pos = np.asarray(pos, dtype=np.float64)
    L = np.broadcast_to(np.asarray(box, dtype=np.float64), (3,))
    n = pos.shape[0]
    F = np.zeros((n, 3))
    W = np.zeros((3, 3))
    hits = 0
    rng = range(-reach, reach + 1)
    for nx, ny, nz in itertools.product(rng, rng, range(-1, 2)):
        shift = np.array([nx * L[0] + nz * dX, ny * L[1], nz * L[2]])
        d = pos[:, None, :] - (pos[None, :, :] + shift)       # r_i - image(r_j)
        r2 = np.einsum("ijk,ijk->ij", d, d)
        mask = r2 < rc * rc
        if nx == 0 and ny == 0 and nz == 0:
            np.fill_diagonal(mask, False)
        if not mask.any():
            continue
        ii, jj = np.nonzero(mask)
        fr = lj_f_over_r(r2[ii, jj], eps, sigma)
        np.add.at(F, ii, fr[:, None] * d[ii, jj])
        hits += ii.size
        # every interacting (i, image j) pair appears twice overall (once from
        # each side), so half of the dyads gives the i<j virial sum
        W += 0.5 * np.einsum("p,pa,pb->ab", fr, d[ii, jj], d[ii, jj])
    return F, W, hits
