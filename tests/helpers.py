"""Small test-side utilities (no GPU, no oracle arithmetic)."""
import numpy as np


def shear_affine(pos, box, dX):
    """Map a configuration that is valid under plain periodic boundaries onto
    the sheared image lattice with offset dX: x -> x + z*dX/Lz (mod Lx).  The
    image above, at z + Lz, then lands exactly dX further along x."""
    L = np.broadcast_to(np.asarray(box, dtype=np.float64), (3,))
    u = np.array(pos, dtype=np.float64)
    u[:, 0] = np.mod(u[:, 0] + u[:, 2] * (dX / L[2]), L[0])
    return u


def le_delta(a, b, box, dX):
    """Difference a - b of two sets of wrapped positions, taken as the
    separation of the nearest images on the sheared lattice with offset dX
    (used to compare positions that may sit on opposite faces)."""
    L = np.broadcast_to(np.asarray(box, dtype=np.float64), (3,))
    d = np.array(a, dtype=np.float64) - np.asarray(b, dtype=np.float64)
    up = d[:, 2] > 0.5 * L[2]
    dn = d[:, 2] < -0.5 * L[2]
    d[up, 2] -= L[2]
    d[up, 0] -= dX
    d[dn, 2] += L[2]
    d[dn, 0] += dX
    d[:, 0] -= L[0] * np.rint(d[:, 0] / L[0])
    d[:, 1] -= L[1] * np.rint(d[:, 1] / L[1])
    return d


def force_errors(f, ref):
    """(global relative L2 error, worst per-particle error scaled by
    max(|F_i|, mean |F|))."""
    f = np.asarray(f)
    ref = np.asarray(ref)
    g = float(np.linalg.norm(f - ref) / np.linalg.norm(ref))
    nr = np.linalg.norm(ref, axis=1)
    scale = np.maximum(nr, nr.mean())
    p = float((np.linalg.norm(f - ref, axis=1) / scale).max())
    return g, p


def flip_resolved_errors(f, ref, ij, fband, inside, rows=None):
    """Force errors once the cut-off decisions of band pairs are taken out.

    A pair whose distance lies within the rounding band of the strict cut-off
    may be counted by a reduced-precision evaluation and not by the FP64
    reference, or the other way round; either is a correct result at that
    precision.  For each particle the subset of its band pairs (ij, pair
    forces fband, `inside` = counted by the reference) that best explains
    f - ref is taken as the tested path's decision, and the rest of the
    difference is its error.

    f, ref: forces of the particles `rows` (all particles when None).
    Returns (global relative L2 error, worst per-particle error scaled by
    max(|F_i|, mean |F|), number of band pairs decided the other way, number
    of band pairs of these particles)."""
    f = np.asarray(f, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    res = f - ref
    row_of = None if rows is None else {int(r): k for k, r in enumerate(rows)}
    by_row = {}
    for k, i in enumerate(np.asarray(ij)[:, 0] if len(ij) else []):
        key = int(i) if row_of is None else row_of.get(int(i))
        if key is None:
            continue
        by_row.setdefault(key, []).append(k)
    flips = 0
    nband = 0
    for row, ks in by_row.items():
        nband += len(ks)
        ks = ks[:12]
        best, best_x = None, None
        for mask in range(1 << len(ks)):
            x = np.array([(mask >> q) & 1 for q in range(len(ks))], dtype=np.float64)
            corr = ((x - inside[ks].astype(np.float64))[:, None] * fband[ks]).sum(axis=0)
            e = np.linalg.norm(res[row] - corr)
            if best is None or e < best:
                best, best_x = e, x
        res[row] -= ((best_x - inside[ks].astype(np.float64))[:, None] * fband[ks]).sum(axis=0)
        flips += int(np.sum(best_x != inside[ks]))
    g = float(np.linalg.norm(res) / np.linalg.norm(ref))
    nr = np.linalg.norm(ref, axis=1)
    scale = np.maximum(nr, nr.mean())
    q = float((np.linalg.norm(res, axis=1) / scale).max())
    return g, q, flips, nband
