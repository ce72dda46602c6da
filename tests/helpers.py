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
