"""TEST INFRASTRUCTURE ONLY: the FP64 CPU oracle for Lees-Edwards shear-flow MD.

Plain, slow and single-threaded.  Only the tests, ``__graft_entry__.smoke()``
and the benchmark's CPU-baseline leg may import this package.  It shares no
code with the CUDA library under ``paper_2109_11083_gb300/``.

The arithmetic lives in ``le_oracle.c`` (compiled with gcc on first use);
``brute.py`` holds an independent numpy image-enumeration force sum used to
pin it.  Every function cites the part of Xu et al. (arXiv 2109.11083) it
follows: Eq. 1 (shear profile), Eq. 4 / Fig. 1 (LE image offset and wrap),
Eq. 5 (Langevin on peculiar velocity), Eqs. 9-11 (LJ, shifted LJ, FENE) and
Eq. 15 (Irving-Kirkwood stress).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "le_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "le_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (no architecture-specific flags)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"],
                   check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(C.Structure):
    _fields_ = [
        ("L", C.c_double * 3),
        ("shear_rate", C.c_double),
        ("rc", C.c_double),
        ("eps", C.c_double),
        ("sigma", C.c_double),
        ("lj_shift", C.c_int),
        ("fene_k", C.c_double),
        ("fene_R0", C.c_double),
        ("mass", C.c_double),
        ("kT", C.c_double),
        ("xi", C.c_double),
        ("dt", C.c_double),
        ("thermostat", C.c_int),
        ("seed", C.c_uint64),
        ("system", C.c_uint64),
        ("nbins", C.c_int),
        ("angle_k", C.c_double),
        ("force_cap", C.c_double),
    ]


class Samples(C.Structure):
    _fields_ = [
        ("nsamples", C.c_int64),
        ("sxz_sum", C.c_double),
        ("stress", C.c_double * 9),
        ("tpec", C.c_double),
        ("epot", C.c_double),
        ("vx_sum", C.POINTER(C.c_double)),
        ("count", C.POINTER(C.c_int64)),
        ("vy2_sum", C.POINTER(C.c_double)),
    ]


OK, BOND_BROKEN, BOX_TOO_SMALL, NONFINITE = 0, 1, 2, 3

_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.ora_dX.restype = C.c_double
            L.ora_dX.argtypes = [C.POINTER(Params), C.c_int64]
            L.ora_vs.restype = C.c_double
            L.ora_vs.argtypes = [C.POINTER(Params), C.c_double]
            L.ora_min_image.restype = None
            L.ora_min_image.argtypes = [C.POINTER(Params), C.c_double, _D, _D, _D]
            L.ora_philox4x64.restype = None
            L.ora_philox4x64.argtypes = [C.POINTER(C.c_uint64)] * 3
            L.ora_noise.restype = None
            L.ora_noise.argtypes = [C.POINTER(Params), C.c_int64, C.c_int64, _D]
            L.ora_pair_uniform.restype = C.c_double
            L.ora_pair_uniform.argtypes = [C.POINTER(Params), C.c_int64, C.c_int64, C.c_int64]
            L.ora_forces.restype = C.c_int
            L.ora_forces.argtypes = [C.POINTER(Params), C.c_double, C.c_int64, _D,
                                     C.c_int64, _I32, C.c_int, _D, _D, _D]
            L.ora_init_forces.restype = C.c_int
            L.ora_init_forces.argtypes = [C.POINTER(Params), C.c_int64, C.c_int64, _D, _D,
                                          C.c_int64, _I32, C.c_int, _D, _D, _D, _D]
            L.ora_run.restype = C.c_int
            L.ora_run.argtypes = [C.POINTER(Params), C.POINTER(C.c_int64), C.c_int64,
                                  C.c_int64, _D, _D, _D, _D, C.c_int64, _I32, C.c_int,
                                  _I32, C.c_int, C.POINTER(Samples)]
            L.ora_forces_on.restype = None
            L.ora_forces_on.argtypes = [C.POINTER(Params), C.c_double, C.c_int64, _D,
                                        C.c_int64, C.POINTER(C.c_int64), _D]
            L.ora_force_error_bound.restype = None
            L.ora_force_error_bound.argtypes = [C.POINTER(Params), C.c_double, C.c_int64, _D,
                                                C.c_int64, _I32, C.c_double, C.c_double, _D]
            L.ora_band_pairs.restype = C.c_int64
            L.ora_band_pairs.argtypes = [C.POINTER(Params), C.c_double, C.c_int64, _D,
                                         C.c_double, C.c_int64, C.POINTER(C.c_int64), _D,
                                         _I32]
            L.ora_observe.restype = C.c_int
            L.ora_observe.argtypes = [C.POINTER(Params), C.c_int64, C.c_int64, _D, _D,
                                      C.c_int64, _I32, C.c_int, _D, _D, _D]
            _lib = L
    return _lib


def params(box, shear_rate, rc, *, eps=1.0, sigma=1.0, lj_shift=1, fene_k=0.0,
           fene_R0=1.5, mass=1.0, kT=1.0, xi=1.0, dt=0.005, thermostat=1,
           seed=0, system=0, nbins=20, angle_k=0.0, force_cap=0.0) -> Params:
    b = np.broadcast_to(np.asarray(box, dtype=np.float64), (3,))
    p = Params()
    p.L = (C.c_double * 3)(*b)
    p.shear_rate, p.rc, p.eps, p.sigma = shear_rate, rc, eps, sigma
    p.lj_shift, p.fene_k, p.fene_R0 = lj_shift, fene_k, fene_R0
    p.mass, p.kT, p.xi, p.dt, p.thermostat = mass, kT, xi, dt, thermostat
    p.seed, p.system, p.nbins = seed, system, nbins
    p.angle_k = angle_k
    p.force_cap = force_cap
    return p


def _dp(a):
    return a.ctypes.data_as(_D)


def _bonds(bonds):
    if bonds is None or len(bonds) == 0:
        return np.zeros((0, 2), dtype=np.int32)
    return np.ascontiguousarray(np.asarray(bonds, dtype=np.int32).reshape(-1, 2))


def dX(p: Params, step: int) -> float:
    """Eq. 4: image offset at integer step `step`."""
    return lib().ora_dX(C.byref(p), step)


def min_image(p: Params, dx_offset: float, ri, rj) -> np.ndarray:
    ri = np.ascontiguousarray(ri, dtype=np.float64)
    rj = np.ascontiguousarray(rj, dtype=np.float64)
    d = np.zeros(3)
    lib().ora_min_image(C.byref(p), dx_offset, _dp(ri), _dp(rj), _dp(d))
    return d


def philox4x64(ctr, key) -> np.ndarray:
    c = (C.c_uint64 * 4)(*[int(x) for x in ctr])
    k = (C.c_uint64 * 2)(*[int(x) for x in key])
    o = (C.c_uint64 * 4)()
    lib().ora_philox4x64(c, k, o)
    return np.array(list(o), dtype=np.uint64)


def noise(p: Params, step: int, gid: int) -> np.ndarray:
    u = np.zeros(3)
    lib().ora_noise(C.byref(p), step, gid, _dp(u))
    return u


def pair_uniform(p: Params, step: int, a: int, b: int) -> float:
    """theta_ij of the DPD random force (Eq. 7): U(-1/2, 1/2), shared by a pair."""
    return lib().ora_pair_uniform(C.byref(p), step, a, b)


def thermostat_forces(p: Params, step: int, pos, vel, bonds=None):
    """(Fc, Ftot) at step for the state (pos, half-step vel): Ftot includes the
    thermostat (Eq. 5, its absolute variant, or DPD of Eqs. 6-8)."""
    s = State(p, pos, vel, bonds=bonds, step=step)
    return s.Fc.copy(), s.Ftot.copy()


def forces(p: Params, dx_offset: float, pos, bonds=None, use_cells=True):
    """Conservative forces (LJ + FENE) at image offset dx_offset.

    Returns (status, F (n,3), W (3,3) = sum_{i<j} r_ij (x) F_ij, epot)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    n = pos.shape[0]
    b = _bonds(bonds)
    F = np.zeros((n, 3))
    W = np.zeros(9)
    e = np.zeros(1)
    st = lib().ora_forces(C.byref(p), dx_offset, n, _dp(pos), b.shape[0],
                          b.ctypes.data_as(_I32), int(use_cells), _dp(F), _dp(W), _dp(e))
    return st, F, W.reshape(3, 3), float(e[0])


def forces_on(p: Params, dx_offset: float, pos, idx) -> np.ndarray:
    """LJ forces on the particles idx only (cell list over all particles)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    ii = np.ascontiguousarray(idx, dtype=np.int64)
    F = np.zeros((ii.size, 3))
    lib().ora_forces_on(C.byref(p), dx_offset, pos.shape[0], _dp(pos), ii.size,
                        ii.ctypes.data_as(C.POINTER(C.c_int64)), _dp(F))
    return F


def force_error_bound(p: Params, dx_offset: float, pos, bonds=None, u: float = 2.0 ** -24,
                      P: float = 1.6) -> np.ndarray:
    """Per-particle first-order bound on the error of forces computed with
    unit roundoff u from reference-relative coordinates (|p| <= P)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    b = _bonds(bonds)
    B = np.zeros(pos.shape[0])
    lib().ora_force_error_bound(C.byref(p), dx_offset, pos.shape[0], _dp(pos), b.shape[0],
                                b.ctypes.data_as(_I32), u, P, _dp(B))
    return B


def band_pairs(p: Params, dx_offset: float, pos, band: float):
    """Ordered pairs within `band` of the LJ cut-off (|r - rc| <= band).

    Returns (ij (m,2) int64, pair force F_ij on i (m,3), inside (m,) bool:
    whether the oracle's strict r < rc test counts the pair)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    cap = 64
    while True:
        ij = np.zeros((cap, 2), dtype=np.int64)
        f = np.zeros((cap, 3))
        inside = np.zeros(cap, dtype=np.int32)
        m = lib().ora_band_pairs(C.byref(p), dx_offset, pos.shape[0], _dp(pos), band, cap,
                                 ij.ctypes.data_as(C.POINTER(C.c_int64)), _dp(f),
                                 inside.ctypes.data_as(_I32))
        if m <= cap:
            return ij[:m], f[:m], inside[:m].astype(bool)
        cap = int(m)


class State:
    """An oracle trajectory: positions, lab-frame velocities, forces, step."""

    def __init__(self, p: Params, pos, vel, bonds=None, step: int = 0, use_cells=True,
                 nbins: int | None = None):
        self.p = p
        self.pos = np.array(pos, dtype=np.float64, order="C", copy=True)
        self.vel = np.array(vel, dtype=np.float64, order="C", copy=True)
        self.n = self.pos.shape[0]
        self.bonds = _bonds(bonds)
        self.step = C.c_int64(step)
        self.use_cells = int(use_cells)
        self.Fc = np.zeros((self.n, 3))
        self.Ftot = np.zeros((self.n, 3))
        self.zimg = np.zeros(self.n, dtype=np.int32)
        nb = p.nbins if nbins is None else nbins
        self.vx_sum = np.zeros(max(nb, 1))
        self.vy2_sum = np.zeros(max(nb, 1))
        self.count = np.zeros(max(nb, 1), dtype=np.int64)
        self.samples = Samples()
        self.samples.vx_sum = _dp(self.vx_sum)
        self.samples.vy2_sum = _dp(self.vy2_sum)
        self.samples.count = self.count.ctypes.data_as(C.POINTER(C.c_int64))
        W = np.zeros(9)
        e = np.zeros(1)
        self.status = lib().ora_init_forces(
            C.byref(p), step, self.n, _dp(self.pos), _dp(self.vel), self.bonds.shape[0],
            self.bonds.ctypes.data_as(_I32), self.use_cells, _dp(self.Fc), _dp(self.Ftot),
            _dp(W), _dp(e))

    def run(self, nsteps: int, sample_every: int = 0) -> int:
        self.status = lib().ora_run(
            C.byref(self.p), C.byref(self.step), nsteps, self.n, _dp(self.pos),
            _dp(self.vel), _dp(self.Fc), _dp(self.Ftot), self.bonds.shape[0],
            self.bonds.ctypes.data_as(_I32), self.use_cells,
            self.zimg.ctypes.data_as(_I32), sample_every, C.byref(self.samples))
        return self.status

    def observe(self):
        """(stress 3x3 of Eq. 15, peculiar temperature, potential energy)."""
        s = np.zeros(9)
        t = np.zeros(1)
        e = np.zeros(1)
        lib().ora_observe(C.byref(self.p), self.step.value, self.n, _dp(self.pos),
                          _dp(self.vel), self.bonds.shape[0],
                          self.bonds.ctypes.data_as(_I32), self.use_cells,
                          _dp(s), _dp(t), _dp(e))
        return s.reshape(3, 3), float(t[0]), float(e[0])

    @property
    def profile(self) -> np.ndarray:
        """Mean lab-frame vx per z bin over the samples taken so far."""
        with np.errstate(invalid="ignore", divide="ignore"):
            return self.vx_sum / self.count

    @property
    def ty_profile(self) -> np.ndarray:
        """T_y per z bin (Sec. 3.1): mean of m vy^2 over the samples."""
        with np.errstate(invalid="ignore", divide="ignore"):
            return self.vy2_sum / self.count

    def density_profile(self, nsamples: int) -> np.ndarray:
        """Number density per z bin (Sec. 3.1): mean count / bin volume."""
        nb = self.count.shape[0]
        L = np.broadcast_to(np.asarray([self.p.L[0], self.p.L[1], self.p.L[2]]), (3,))
        return self.count / (nsamples * L[0] * L[1] * L[2] / nb)
