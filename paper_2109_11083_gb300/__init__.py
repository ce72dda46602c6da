"""GB300 (sm_103a) Lees-Edwards shear-flow molecular dynamics.

A thin ctypes binding of the C ABI declared in ``include/le.h``: every
function ``le_*`` below has the name of the C entry point it marshals
arguments for, and every step of the method runs in the library's CUDA
kernels.  The library is built in-tree by ``paper_2109_11083_gb300.build``;
importing works without it, but the first call raises if it is missing (there
is no CPU fallback).

The method follows Xu et al., "Implementation and Parallel Optimization of
the Lees-Edwards Boundary Condition in ESPResSo++" (arXiv 2109.11083): the
sheared periodic images of Eq. 4 / Fig. 1, LJ/WCA and FENE forces (Eqs. 9-11),
the Langevin thermostat on peculiar velocities (Eq. 5) and the Irving-Kirkwood
stress for the viscosity (Eqs. 14-15).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

LE_OK = 0
STATUS = {
    0: "LE_OK", 1: "LE_ERR_INVALID_ARG", 2: "LE_ERR_CUDA", 3: "LE_ERR_OOM",
    4: "LE_ERR_BOX_TOO_SMALL", 5: "LE_ERR_BOND_BROKEN", 6: "LE_ERR_NONFINITE",
    7: "LE_ERR_CAPACITY", 8: "LE_ERR_TIMEOUT", 9: "LE_ERR_STATE", 10: "LE_ERR_RANGE",
}
LE_FP64, LE_FP32 = 0, 1
LE_THERMO_NONE, LE_THERMO_PECULIAR, LE_THERMO_ABSOLUTE, LE_THERMO_DPD = 0, 1, 2, 3


class LEError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class le_params(C.Structure):
    _fields_ = [
        ("eps", C.c_double), ("sigma", C.c_double), ("mass", C.c_double),
        ("kT", C.c_double), ("xi", C.c_double), ("dt", C.c_double),
        ("lj_shift", C.c_int), ("thermostat", C.c_int),
        ("fene_k", C.c_double), ("fene_R0", C.c_double),
        ("precision", C.c_int),
        ("seed", C.c_uint64), ("system_id", C.c_uint64),
        ("sample_every", C.c_int), ("profile_bins", C.c_int),
        ("angle_k", C.c_double),
        ("force_cap", C.c_double),
    ]


class le_counters(C.Structure):
    _fields_ = [
        ("step", C.c_int64), ("particles", C.c_int64), ("rebuilds", C.c_int64),
        ("image_rebuilds", C.c_int64), ("list_capacity", C.c_int64),
        ("list_max", C.c_int64), ("cells", C.c_int64 * 3), ("dX", C.c_double),
        ("list_mean", C.c_double), ("force_threads", C.c_int32), ("list_threads", C.c_int32),
    ]


_lib = None
_lock = threading.Lock()
_D = C.POINTER(C.c_double)
_P = C.c_void_p


def library_path() -> str:
    return _build.LIB


def lib():
    """The loaded CUDA library.  Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(
                    f"the CUDA library {path} is not built; run "
                    "`python -c 'import __graft_entry__ as g; g.build()'` first")
            L = C.CDLL(path)
            sig = {
                "le_default_params": (None, [C.POINTER(le_params)]),
                "le_create": (C.c_int, [_D, C.c_double, C.c_double, C.c_double,
                                        C.POINTER(le_params), _P, C.POINTER(_P)]),
                "le_set_bonds": (C.c_int, [_P, C.c_int64, C.POINTER(C.c_int32)]),
                "le_set_particles": (C.c_int, [_P, C.c_int64, _D, _D]),
                "le_step": (C.c_int, [_P, C.c_int64]),
                "le_step_profiled": (C.c_int, [_P, C.c_int64, _D, _D, _D]),
                "le_forces": (C.c_int, [_P, _D]),
                "le_positions": (C.c_int, [_P, _D, _D]),
                "le_stress": (C.c_int, [_P, _D, _D, C.POINTER(C.c_int64)]),
                "le_velocity_profile": (C.c_int, [_P, C.c_int, _D, C.POINTER(C.c_int64)]),
                "le_profiles": (C.c_int, [_P, C.c_int, _D, _D, _D, C.POINTER(C.c_int64)]),
                "le_temperature": (C.c_int, [_P, _D]),
                "le_reset_samples": (C.c_int, [_P]),
                "le_get_counters": (C.c_int, [_P, C.POINTER(le_counters)]),
                "le_set_launch": (C.c_int, [_P, C.c_int, C.c_int]),
                "le_tune": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), _D]),
                "le_batch_tune": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), _D]),
                "le_get_state": (C.c_int, [_P, _P, C.POINTER(C.c_size_t)]),
                "le_set_state": (C.c_int, [_P, _P, C.c_size_t]),
                "le_set_eager": (C.c_int, [_P, C.c_int]),
                "le_estimate_device_bytes": (C.c_int, [_D, C.c_double, C.c_double, C.c_double,
                                                       C.POINTER(le_params), C.c_int64,
                                                       C.c_int64, C.POINTER(C.c_size_t)]),
                "le_batch_create": (C.c_int, [C.c_size_t, _P, C.POINTER(_P)]),
                "le_batch_add": (C.c_int, [_P, _P]),
                "le_batch_remove": (C.c_int, [_P, _P]),
                "le_batch_step": (C.c_int, [_P, C.c_int64]),
                "le_batch_destroy": (C.c_int, [_P]),
                "le_batch_last_error": (C.c_char_p, [_P]),
                "le_forces_noalloc": (C.c_int, [_D, C.c_double, C.c_double, C.c_double,
                                                C.POINTER(le_params), C.c_int64, C.c_int64,
                                                _D, _D, _P]),
                "le_sort_cell_keys": (C.c_int, [C.c_int64, C.POINTER(C.c_uint32), C.c_int,
                                                C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                                                _P]),
                "le_fp32_peak": (C.c_int, [_D, _D]),
                "le_wait_selftest": (C.c_int, [_P, _D]),
                "le_destroy": (C.c_int, [_P]),
                "le_last_error": (C.c_char_p, [_P]),
                "le_status_string": (C.c_char_p, [C.c_int]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def exported_symbols() -> list[str]:
    """Names of the C entry points this binding expects the library to export."""
    return ["le_default_params", "le_create", "le_set_bonds", "le_set_particles", "le_step",
            "le_step_profiled", "le_forces", "le_positions", "le_stress",
            "le_velocity_profile", "le_profiles", "le_temperature", "le_reset_samples", "le_get_counters",
            "le_set_launch", "le_tune", "le_batch_tune",
            "le_get_state", "le_set_state", "le_set_eager", "le_destroy", "le_last_error",
            "le_status_string", "le_forces_noalloc", "le_estimate_device_bytes",
            "le_sort_cell_keys",
            "le_batch_create", "le_batch_add", "le_batch_remove", "le_batch_step",
            "le_batch_destroy", "le_batch_last_error"]


def _check(h, st: int):
    if st != LE_OK:
        msg = lib().le_last_error(h).decode(errors="replace") if h else ""
        raise LEError(st, msg)


def _f64(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(getattr(stream, "cuda_stream"))  # torch.cuda.Stream


# ---------------------------------------------------------------- C-ABI names
def le_default_params() -> le_params:
    p = le_params()
    lib().le_default_params(C.byref(p))
    return p


def le_create(box, shear_rate: float, rc: float, skin: float, params: le_params | None = None,
              stream=None) -> int:
    p = params if params is not None else le_default_params()
    b = _f64(np.broadcast_to(np.asarray(box, dtype=np.float64), (3,)))
    h = _P()
    st = lib().le_create(b.ctypes.data_as(_D), float(shear_rate), float(rc), float(skin),
                         C.byref(p), _stream_handle(stream), C.byref(h))
    _check(None, st)
    return h.value


def le_set_bonds(h: int, pairs) -> None:
    a = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    _check(h, lib().le_set_bonds(h, a.shape[0], a.ctypes.data_as(C.POINTER(C.c_int32))))


def le_set_particles(h: int, pos, vel) -> None:
    p = _f64(pos, (-1, 3))
    v = _f64(vel, (-1, 3))
    if p.shape != v.shape:
        raise ValueError("pos and vel must have the same shape")
    _check(h, lib().le_set_particles(h, p.shape[0], p.ctypes.data_as(_D), v.ctypes.data_as(_D)))


def le_step(h: int, nsteps: int) -> None:
    _check(h, lib().le_step(h, int(nsteps)))


def le_step_profiled(h: int, nsteps: int) -> tuple[float, float, float]:
    """(pair-force kernel ms, integrate kernel ms, whole graph ms), summed over
    the nsteps of one graph launch."""
    f, i, t = C.c_double(), C.c_double(), C.c_double()
    _check(h, lib().le_step_profiled(h, int(nsteps), C.byref(f), C.byref(i), C.byref(t)))
    return f.value, i.value, t.value


def le_forces(h: int, n: int, out: np.ndarray | None = None) -> np.ndarray:
    o = np.empty((n, 3)) if out is None else out
    _check(h, lib().le_forces(h, o.ctypes.data_as(_D)))
    return o


def le_positions(h: int, n: int, pos: np.ndarray | None = None, vel: np.ndarray | None = None):
    p = np.empty((n, 3)) if pos is None else pos
    v = np.empty((n, 3)) if vel is None else vel
    _check(h, lib().le_positions(h, p.ctypes.data_as(_D), v.ctypes.data_as(_D)))
    return p, v


def le_stress(h: int, instantaneous: bool = True):
    """(3x3 instantaneous Eq. 15 tensor or None, mean sigma_xz, samples)."""
    s = np.empty(9)
    xz = C.c_double()
    ns = C.c_int64()
    _check(h, lib().le_stress(h, s.ctypes.data_as(_D) if instantaneous else None,
                              C.byref(xz), C.byref(ns)))
    return (s.reshape(3, 3) if instantaneous else None), xz.value, ns.value


def le_velocity_profile(h: int, nbins: int):
    vx = np.empty(nbins)
    cnt = np.empty(nbins, dtype=np.int64)
    _check(h, lib().le_velocity_profile(h, nbins, vx.ctypes.data_as(_D),
                                        cnt.ctypes.data_as(C.POINTER(C.c_int64))))
    return vx, cnt


def le_profiles(h: int, nbins: int):
    """(vx mean, T_y, density, counts) per z bin over the samples (Sec. 3.1)."""
    vx, ty, rho = np.empty(nbins), np.empty(nbins), np.empty(nbins)
    cnt = np.empty(nbins, dtype=np.int64)
    _check(h, lib().le_profiles(h, nbins, vx.ctypes.data_as(_D), ty.ctypes.data_as(_D),
                                rho.ctypes.data_as(_D), cnt.ctypes.data_as(C.POINTER(C.c_int64))))
    return vx, ty, rho, cnt


def le_temperature(h: int) -> float:
    t = C.c_double()
    _check(h, lib().le_temperature(h, C.byref(t)))
    return t.value


def le_reset_samples(h: int) -> None:
    _check(h, lib().le_reset_samples(h))


def le_get_counters(h: int) -> dict:
    c = le_counters()
    _check(h, lib().le_get_counters(h, C.byref(c)))
    return dict(step=c.step, particles=c.particles, rebuilds=c.rebuilds,
                image_rebuilds=c.image_rebuilds, list_capacity=c.list_capacity,
                list_max=c.list_max, cells=tuple(c.cells), dX=c.dX, list_mean=c.list_mean,
                force_threads=c.force_threads, list_threads=c.list_threads)


def le_get_state(h: int) -> bytes:
    n = C.c_size_t()
    _check(h, lib().le_get_state(h, None, C.byref(n)))
    buf = C.create_string_buffer(n.value)
    _check(h, lib().le_get_state(h, C.cast(buf, _P), C.byref(n)))
    return buf.raw[: n.value]


def le_set_state(h: int, blob: bytes) -> None:
    buf = C.create_string_buffer(blob, len(blob))
    _check(h, lib().le_set_state(h, C.cast(buf, _P), len(blob)))


def le_set_eager(h: int, eager: bool) -> None:
    _check(h, lib().le_set_eager(h, 1 if eager else 0))


def le_forces_noalloc(box, shear_rate: float, rc: float, skin: float, params: le_params,
                      step: int, pos, stream=None) -> np.ndarray:
    """Forces at `pos` (image offset of step `step`) without any device
    allocation: for callers that must not allocate device memory."""
    b = _f64(np.broadcast_to(np.asarray(box, dtype=np.float64), (3,)))
    p = _f64(pos, (-1, 3))
    out = np.empty_like(p)
    st = lib().le_forces_noalloc(b.ctypes.data_as(_D), float(shear_rate), float(rc), float(skin),
                                 C.byref(params), int(step), p.shape[0], p.ctypes.data_as(_D),
                                 out.ctypes.data_as(_D), _stream_handle(stream))
    _check(None, st)
    return out


def le_sort_cell_keys(keys, bits: int, stream=None):
    """(order, sorted keys) of the library's stable radix sort of cell keys."""
    k = np.ascontiguousarray(keys, dtype=np.uint32)
    order = np.empty_like(k)
    out = np.empty_like(k)
    u32 = C.POINTER(C.c_uint32)
    st = lib().le_sort_cell_keys(k.size, k.ctypes.data_as(u32), int(bits),
                                 order.ctypes.data_as(u32), out.ctypes.data_as(u32),
                                 _stream_handle(stream))
    _check(None, st)
    return order, out


def le_fp32_peak():
    """(scalar, paired) FP32 FMA throughput of the current device, TFLOP/s."""
    a, b = C.c_double(), C.c_double()
    _check(None, lib().le_fp32_peak(C.byref(a), C.byref(b)))
    return a.value, b.value


def le_wait_selftest(stream=None):
    """(status, ms) of the bounded-wait self-test; status LE_ERR_TIMEOUT (8)
    is the expected outcome."""
    ms = C.c_double()
    st = lib().le_wait_selftest(_stream_handle(stream), C.byref(ms))
    return st, ms.value


def le_estimate_device_bytes(box, shear_rate: float, rc: float, skin: float, params: le_params,
                             n: int, nbonds: int = 0) -> int:
    b = _f64(np.broadcast_to(np.asarray(box, dtype=np.float64), (3,)))
    out = C.c_size_t()
    _check(None, lib().le_estimate_device_bytes(b.ctypes.data_as(_D), float(shear_rate), float(rc),
                                                float(skin), C.byref(params), int(n), int(nbonds),
                                                C.byref(out)))
    return out.value


def _bcheck(b, st: int):
    if st != LE_OK:
        msg = lib().le_batch_last_error(b).decode(errors="replace") if b else ""
        raise LEError(st, msg)


def le_batch_create(budget_bytes: int = 0, stream=None) -> int:
    h = _P()
    _bcheck(None, lib().le_batch_create(int(budget_bytes), _stream_handle(stream), C.byref(h)))
    return h.value


def le_batch_add(b: int, h: int) -> None:
    _bcheck(b, lib().le_batch_add(b, h))


def le_batch_remove(b: int, h: int) -> None:
    _bcheck(b, lib().le_batch_remove(b, h))


def le_batch_step(b: int, nsteps: int) -> None:
    _bcheck(b, lib().le_batch_step(b, int(nsteps)))


def le_batch_tune(b: int, steps_per_trial: int = 32):
    """The batch autotuner: (force threads, list threads, ms per batch step)."""
    f, l, ms = C.c_int(), C.c_int(), C.c_double()
    _bcheck(b, lib().le_batch_tune(b, int(steps_per_trial), C.byref(f), C.byref(l), C.byref(ms)))
    return f.value, l.value, ms.value


def le_set_launch(h: int, force_threads: int, list_threads: int) -> None:
    _check(h, lib().le_set_launch(h, int(force_threads), int(list_threads)))


def le_tune(h: int, steps_per_trial: int = 32):
    """The autotuner: (force threads, list threads, ms per step) it chose."""
    f, l, ms = C.c_int(), C.c_int(), C.c_double()
    _check(h, lib().le_tune(h, int(steps_per_trial), C.byref(f), C.byref(l), C.byref(ms)))
    return f.value, l.value, ms.value


def le_batch_destroy(b: int) -> None:
    _bcheck(None, lib().le_batch_destroy(b))


def le_destroy(h: int) -> None:
    _check(None, lib().le_destroy(h))


# ---------------------------------------------------------------- convenience
class Sim:
    """One sheared box resident on the GPU (a handle of the C ABI)."""

    def __init__(self, box, shear_rate, rc, skin, *, stream=None, **params):
        p = le_default_params()
        for k, v in params.items():
            if not hasattr(p, k):
                raise TypeError(f"unknown parameter {k}")
            setattr(p, k, v)
        self.params = p
        self.box = np.broadcast_to(np.asarray(box, dtype=np.float64), (3,)).copy()
        self.shear_rate = float(shear_rate)
        self.h = le_create(self.box, shear_rate, rc, skin, p, stream)
        self.n = 0

    def set_bonds(self, pairs):
        le_set_bonds(self.h, pairs)

    def set_particles(self, pos, vel):
        pos = _f64(pos, (-1, 3))
        le_set_particles(self.h, pos, vel)
        self.n = pos.shape[0]

    def step(self, nsteps):
        le_step(self.h, nsteps)

    def step_profiled(self, nsteps):
        return le_step_profiled(self.h, nsteps)

    def forces(self):
        return le_forces(self.h, self.n)

    def positions(self):
        return le_positions(self.h, self.n)

    def stress(self, instantaneous=True):
        return le_stress(self.h, instantaneous)

    def velocity_profile(self):
        return le_velocity_profile(self.h, self.params.profile_bins)

    def profiles(self):
        """(vx mean, T_y, density, counts) per z bin (Sec. 3.1, Fig. 3)."""
        return le_profiles(self.h, self.params.profile_bins)

    def temperature(self):
        return le_temperature(self.h)

    def reset_samples(self):
        le_reset_samples(self.h)

    def counters(self):
        return le_get_counters(self.h)

    def set_launch(self, force_threads: int, list_threads: int):
        le_set_launch(self.h, force_threads, list_threads)

    def tune(self, steps_per_trial: int = 32):
        """Autotunes the launch shapes (results unchanged); returns the choice."""
        return le_tune(self.h, steps_per_trial)

    def get_state(self):
        return le_get_state(self.h)

    def set_state(self, blob):
        le_set_state(self.h, blob)

    def set_eager(self, eager=True):
        le_set_eager(self.h, eager)

    def close(self):
        if self.h:
            le_destroy(self.h)
            self.h = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many handles advanced together by one graph launch per 16 steps."""

    def __init__(self, budget_bytes: int = 0, stream=None):
        self.b = le_batch_create(budget_bytes, stream)
        self.members = []

    def add(self, sim: Sim):
        le_batch_add(self.b, sim.h)
        self.members.append(sim)

    def remove(self, sim: Sim):
        le_batch_remove(self.b, sim.h)
        self.members.remove(sim)

    def step(self, nsteps: int):
        le_batch_step(self.b, nsteps)

    def tune(self, steps_per_trial: int = 32):
        """Autotunes the members' launch shapes on the whole batch (results
        unchanged); returns (force threads, list threads, ms per step)."""
        return le_batch_tune(self.b, steps_per_trial)

    def close(self):
        if self.b:
            le_batch_destroy(self.b)
            self.b = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
