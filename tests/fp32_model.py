"""Test-side model of a reduced-precision LJ force evaluation (numpy float32).

An FP32 evaluation of the LJ pair forces (Eqs. 9-10) from reference-relative
coordinates, written independently of both the CUDA library and the FP64
oracle, so that it can pin the oracle's first-order rounding bound
(``oracle.force_error_bound``) from the outside:

- every particle stores its displacement p from the centre of a reference cell
  of a grid of edge >= rc + skin, rounded to float32; the reference cell may
  be a neighbour of the particle's current cell (the particle has drifted
  since the grid was built), so |p| reaches half a cell edge plus half the
  skin;
- a pair's separation is the float32 difference p_i - p_j plus the offset
  between the two cell centres, itself rounded to float32 (for a pair across
  the top/bottom face the LE image offset dX of Eq. 4 is part of it);
- r^2, 1/r^2 and the force factor are float32 operations, and each particle's
  force is a sequential float32 sum over its pairs.

Which pairs interact, and the offsets between references, come from the FP64
minimum image here; the model measures rounding only.
"""
from __future__ import annotations

import math

import numpy as np

F32 = np.float32


def cell_grid(box, edge):
    """Cells per dimension and cell edge of a grid of edge >= `edge`."""
    L = np.broadcast_to(np.asarray(box, dtype=np.float64), (3,))
    nc = np.maximum(1, np.floor(L / edge)).astype(np.int64)
    return nc, L / nc


def ordered_pairs(pos, box, dX, rmax):
    """Every ordered pair (i, j != i) with an LE minimum-image separation below
    rmax: (i, j, d (FP64, r_i - image of r_j), image z index of j)."""
    pos = np.asarray(pos, dtype=np.float64)
    L = np.broadcast_to(np.asarray(box, dtype=np.float64), (3,))
    n = pos.shape[0]
    out_i, out_j, out_d, out_nz = [], [], [], []
    for i0 in range(0, n, 256):
        blk = pos[i0:i0 + 256]
        d = blk[:, None, :] - pos[None, :, :]
        nz = np.where(d[..., 2] > 0.5 * L[2], 1, np.where(d[..., 2] < -0.5 * L[2], -1, 0))
        d[..., 2] -= nz * L[2]
        d[..., 0] -= nz * dX
        d[..., 0] -= L[0] * np.rint(d[..., 0] / L[0])
        d[..., 1] -= L[1] * np.rint(d[..., 1] / L[1])
        r2 = np.einsum("ijk,ijk->ij", d, d)
        m = r2 < rmax * rmax
        ii = np.arange(blk.shape[0])
        m[ii, i0 + ii] = False
        a, b = np.nonzero(m)
        out_i.append(a + i0)
        out_j.append(b)
        out_d.append(d[a, b])
        out_nz.append(nz[a, b])
    return (np.concatenate(out_i), np.concatenate(out_j), np.concatenate(out_d),
            np.concatenate(out_nz))


def reference_cells(pos, box, edge, drift, seed=0):
    """A reference cell per particle: the cell of the particle displaced by a
    random vector of length <= drift (a grid built before the particle moved).
    Returns (displacement p from the reference centre (FP64), largest |p_a|)."""
    pos = np.asarray(pos, dtype=np.float64)
    nc, lc = cell_grid(box, edge)
    g = np.random.default_rng(seed)
    u = g.normal(size=pos.shape)
    u *= (drift * g.uniform(size=(pos.shape[0], 1)) ** (1 / 3)) / np.linalg.norm(u, axis=1,
                                                                               keepdims=True)
    c = np.floor((pos + u) / lc).astype(np.int64)   # unwrapped cell index
    p = pos - (c + 0.5) * lc
    return p, float(np.abs(p).max())


def f32_forces(pos, box, dX, rc, edge, drift=0.0, seed=0, eps=1.0, sigma=1.0):
    """FP32 model forces and the pairs it used.

    Returns (F (n,3) in float64, pairs tuple, r2 of each pair in float32,
    largest reference-relative coordinate P)."""
    pos = np.asarray(pos, dtype=np.float64)
    n = pos.shape[0]
    i, j, d64, nz = ordered_pairs(pos, box, dX, rc + 0.5)
    p, P = reference_cells(pos, box, edge, drift, seed)
    # offset between the two references for this image: d = p_i - p_j + off
    off = d64 - (p[i] - p[j])
    pf = p.astype(F32)
    d = (pf[i] - pf[j]) + off.astype(F32)             # float32 throughout
    r2 = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2]
    s2 = F32(sigma * sigma) / r2
    s6 = s2 * s2 * s2
    fr = F32(24.0 * eps) * (F32(2.0) * s6 * s6 - s6) / r2
    fr = np.where(r2 < F32(rc * rc), fr, F32(0.0))
    F = np.zeros((n, 3), dtype=F32)
    # sequential float32 sum per particle, pairs in index order
    order = np.lexsort((j, i))
    for a in range(3):
        np.add.at(F[:, a], i[order], (fr * d[:, a])[order])
    return F.astype(np.float64), (i, j, d64, nz), r2, P


def separation_errors(pos, box, dX, rc, edge, drift=0.0, seed=0):
    """Per-pair |d_float32 - d_FP64| (worst component) and r, for pairs within rc."""
    pos = np.asarray(pos, dtype=np.float64)
    i, j, d64, nz = ordered_pairs(pos, box, dX, rc)
    p, P = reference_cells(pos, box, edge, drift, seed)
    off = d64 - (p[i] - p[j])
    pf = p.astype(F32)
    d = ((pf[i] - pf[j]) + off.astype(F32)).astype(np.float64)
    return np.abs(d - d64).max(axis=1), np.linalg.norm(d64, axis=1), P
