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
