"""respa3b Python binding: argument marshalling over the C ABI of librespa3b.so.

Every function below calls the entry point of the same name declared in
include/respa3b.h; all computation happens in the library's CUDA kernels
(sm_103a).  There is no CPU fallback: importing works anywhere, but
``load()`` raises when the compiled library or a CUDA device is missing.

Arrays are numpy float64 of shape (n, 3) in the caller's particle order.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build_lib

MD_FP32 = 0
MD_FP64 = 1
MD_DEFERRED = 0x100

STATUS = {0: "MD_OK", -1: "MD_ERR_ARG", -2: "MD_ERR_OOM", -3: "MD_ERR_BOX_TOO_SMALL", -4: "MD_ERR_NONFINITE",
          -5: "MD_ERR_DEVICE_TIMEOUT", -6: "MD_ERR_CUDA", -7: "MD_ERR_STATE", -8: "MD_ERR_CAPACITY",
          -9: "MD_ERR_CANCELLED"}


class MDError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} {detail}".strip())


class md_stats(ctypes.Structure):
    _fields_ = [("triplets_last", ctypes.c_uint64), ("triplets_total", ctypes.c_uint64),
                ("atm_evals", ctypes.c_uint64), ("lj_evals", ctypes.c_uint64), ("outer_steps", ctypes.c_uint64),
                ("replays", ctypes.c_uint64), ("guard_rechecks", ctypes.c_uint64), ("atm_ms_total", ctypes.c_double),
                ("atm_timed", ctypes.c_uint64), ("max_cell_count", ctypes.c_int32),
                ("cells_per_side", ctypes.c_int32), ("atm_kernel", ctypes.c_int32), ("atm_bases_per_warp", ctypes.c_int32),
                ("near_triplets_last", ctypes.c_uint64), ("lj_block", ctypes.c_int32), ("list_warps", ctypes.c_int32),
                ("tuned_from_cache", ctypes.c_int32), ("lj_kernel", ctypes.c_int32),
                ("lj_team", ctypes.c_int32), ("reserved_", ctypes.c_int32)]


_lib = None
_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_I64 = ctypes.c_int64
_U64P = ctypes.POINTER(ctypes.c_uint64)

# name -> (restype, argtypes); every symbol declared in include/respa3b.h
SIGNATURES = {
    "md_create_system": (_I, [ctypes.POINTER(_P), _I64, _D, _P, _P, _D, _I, _P]),
    "md_set_potentials": (_I, [_P, _D, _D, _D, _D, _D]),
    "md_set_skin": (_I, [_P, _D]),
    "md_respa_step": (_I, [_P, _I, _I, _D]),
    "md_get_forces": (_I, [_P, _P, _P]),
    "md_get_energy": (_I, [_P, _P, _P, _P, _P]),
    "md_get_rdf": (_I, [_P, _I, _D, _P]),
    "md_get_state": (_I, [_P, _P, _P]),
    "md_set_state": (_I, [_P, _P, _P]),
    "md_get_stats": (_I, [_P, ctypes.POINTER(md_stats)]),
    "md_set_profiling": (_I, [_P, _I]),
    "md_set_atm_kernel": (_I, [_P, _I]),
    "md_set_lj_kernel": (_I, [_P, _I]),
    "md_batch_set_limits": (_I, [_P, ctypes.c_int64]),
    "md_inject_copy_shortfall": (_I, [_P, _I]),
    "md_set_shapes": (_I, [_P, _I, _I, _I]),
    "md_set_distance_classes": (_I, [_P, _D, _I]),
    "md_get_near_forces": (_I, [_P, _P]),
    "md_get_info": (_I, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_D), ctypes.POINTER(_I)]),
    "md_get_memory": (_I, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    "md_destroy_system": (_I, [_P]),
    "md_status_string": (ctypes.c_char_p, [_I]),
    "md_last_error": (ctypes.c_char_p, []),
    "md_batch_create": (_I, [ctypes.POINTER(_P), ctypes.c_size_t]),
    "md_batch_submit": (_I, [_P, _P, _I, _I, _D, _U64P]),
    "md_batch_run": (_I, [_P, _I]),
    "md_batch_poll": (_I, [_P, ctypes.c_uint64, ctypes.POINTER(_I)]),
    "md_batch_latency": (_I, [_P, ctypes.c_uint64, _P, ctypes.POINTER(_I)]),
    "md_batch_pending": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "md_batch_cycles": (_I, [_P, _U64P, _U64P]),
    "md_batch_cancel": (_I, [_P, ctypes.c_uint64]),
    "md_batch_destroy": (_I, [_P]),
    "md_atm_direct": (_I, [_P, _I64, _D, _I, _P, _P, _P]),
    "md_measure_fma_peak": (_I, [_I, _D, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "md_atm_forces_noalloc": (_I, [_P, _I64, _D, _D, _D, _P, ctypes.POINTER(_D), _U64P, _P]),
}


def library_path() -> str:
    return build_lib.LIB


def load(build_if_missing: bool = True):
    """Load librespa3b.so (building it in-tree if absent).  Raises if it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"{path} is missing: run __graft_entry__.build() first")
        build_lib.build()
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(st: int, where: str):
    if st != 0:
        detail = ""
        try:
            detail = (_lib.md_last_error() or b"").decode()
        except Exception:
            pass
        raise MDError(st, where, detail)


def _arr(x, n):
    a = np.ascontiguousarray(x, dtype=np.float64)
    if a.shape != (n, 3):
        raise ValueError(f"expected shape ({n}, 3), got {a.shape}")
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


# ------------------------------------------------------------ same-name wrappers

def md_create_system(pos, box_L: float, vel=None, mass: float = 1.0, precision: int = MD_FP32, stream=None):
    lib = load()
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    n = pos.shape[0]
    pos = _arr(pos, n)
    vel = None if vel is None else _arr(vel, n)
    h = _P()
    st = lib.md_create_system(ctypes.byref(h), n, float(box_L), _ptr(pos), _ptr(vel), float(mass), int(precision),
                              None if stream is None else ctypes.c_void_p(int(stream)))
    _check(st, "md_create_system")
    return h


def md_set_potentials(h, eps=1.0, sigma=1.0, rc_pair=2.5, nu=0.0, rc_triplet=2.5):
    _check(load().md_set_potentials(h, eps, sigma, rc_pair, nu, rc_triplet), "md_set_potentials")


def md_set_skin(h, skin: float):
    _check(load().md_set_skin(h, skin), "md_set_skin")


def md_respa_step(h, n_outer: int, k_inner: int, dt_outer: float):
    _check(load().md_respa_step(h, int(n_outer), int(k_inner), float(dt_outer)), "md_respa_step")


def md_get_info(h):
    n, L, p = _I64(), _D(), _I()
    _check(load().md_get_info(h, ctypes.byref(n), ctypes.byref(L), ctypes.byref(p)), "md_get_info")
    return int(n.value), float(L.value), int(p.value)


def md_get_memory(h) -> int:
    """Device bytes the handle holds (deferred: will hold once resident)."""
    b = ctypes.c_size_t()
    _check(load().md_get_memory(h, ctypes.byref(b)), "md_get_memory")
    return int(b.value)


def md_get_forces(h, f2=True, f3=True):
    n = md_get_info(h)[0]
    a2 = np.empty((n, 3)) if f2 else None
    a3 = np.empty((n, 3)) if f3 else None
    _check(load().md_get_forces(h, _ptr(a2), _ptr(a3)), "md_get_forces")
    return a2, a3


def md_get_energy(h):
    ek, u2, u3, w = _D(), _D(), _D(), _D()
    _check(load().md_get_energy(h, ctypes.byref(ek), ctypes.byref(u2), ctypes.byref(u3), ctypes.byref(w)),
           "md_get_energy")
    return ek.value, u2.value, u3.value, w.value


def md_get_rdf(h, nbins: int, r_max: float) -> np.ndarray:
    counts = np.zeros(int(nbins), dtype=np.uint64)
    _check(load().md_get_rdf(h, int(nbins), float(r_max), _ptr(counts)), "md_get_rdf")
    return counts


def md_get_state(h, pos_out=None, vel_out=None):
    n = md_get_info(h)[0]
    pos = np.empty((n, 3)) if pos_out is None else pos_out
    vel = np.empty((n, 3)) if vel_out is None else vel_out
    _check(load().md_get_state(h, _ptr(pos), _ptr(vel)), "md_get_state")
    return pos, vel


def md_set_state(h, pos=None, vel=None):
    n = md_get_info(h)[0]
    pos = None if pos is None else _arr(pos, n)
    vel = None if vel is None else _arr(vel, n)
    _check(load().md_set_state(h, _ptr(pos), _ptr(vel)), "md_set_state")


def md_get_stats(h) -> dict:
    s = md_stats()
    _check(load().md_get_stats(h, ctypes.byref(s)), "md_get_stats")
    return {k: getattr(s, k) for k, _ in md_stats._fields_}


def md_set_profiling(h, on: bool):
    _check(load().md_set_profiling(h, 1 if on else 0), "md_set_profiling")


def md_set_atm_kernel(h, variant: int):
    _check(load().md_set_atm_kernel(h, int(variant)), "md_set_atm_kernel")


def md_set_lj_kernel(h, variant: int):
    _check(load().md_set_lj_kernel(h, int(variant)), "md_set_lj_kernel")


def md_inject_copy_shortfall(h, nbytes: int):
    _check(load().md_inject_copy_shortfall(h, int(nbytes)), "md_inject_copy_shortfall")


def md_set_shapes(h, lj_block: int = 0, list_warps: int = 0, rot_bases_per_warp: int = 0):
    _check(load().md_set_shapes(h, int(lj_block), int(list_warps), int(rot_bases_per_warp)), "md_set_shapes")


def md_set_distance_classes(h, r_a: float, s_near: int):
    _check(load().md_set_distance_classes(h, float(r_a), int(s_near)), "md_set_distance_classes")


def md_get_near_forces(h, out=None):
    n = md_get_info(h)[0]
    f = np.empty((n, 3)) if out is None else out
    _check(load().md_get_near_forces(h, _ptr(f)), "md_get_near_forces")
    return f


def md_destroy_system(h):
    if h:
        _check(load().md_destroy_system(h), "md_destroy_system")


def md_status_string(st: int) -> str:
    return load().md_status_string(int(st)).decode()


def md_batch_create(hbm_budget_bytes: int = 0):
    h = _P()
    _check(load().md_batch_create(ctypes.byref(h), int(hbm_budget_bytes)), "md_batch_create")
    return h


def md_batch_set_limits(b, max_resident_particles: int):
    _check(load().md_batch_set_limits(b, int(max_resident_particles)), "md_batch_set_limits")


def md_batch_submit(b, sys_h, n_outer: int, k_inner: int, dt_outer: float) -> int:
    t = ctypes.c_uint64()
    _check(load().md_batch_submit(b, sys_h, int(n_outer), int(k_inner), float(dt_outer), ctypes.byref(t)),
           "md_batch_submit")
    return int(t.value)


def md_batch_run(b, max_ticks: int = 0):
    _check(load().md_batch_run(b, int(max_ticks)), "md_batch_run")


def md_batch_poll(b, ticket: int) -> bool:
    d = _I()
    _check(load().md_batch_poll(b, ctypes.c_uint64(ticket), ctypes.byref(d)), "md_batch_poll")
    return bool(d.value)


def md_batch_latency(b, ticket: int, cap: int = 4096) -> np.ndarray:
    """Per-outer-step latencies (ms, device clock) of a ticket's request."""
    buf = np.zeros(cap)
    c = _I(cap)
    _check(load().md_batch_latency(b, ctypes.c_uint64(ticket), _ptr(buf), ctypes.byref(c)), "md_batch_latency")
    return buf[:c.value].copy()


def md_batch_pending(b):
    q, r = _I(), _I()
    _check(load().md_batch_pending(b, ctypes.byref(q), ctypes.byref(r)), "md_batch_pending")
    return q.value, r.value


def md_batch_cycles(b):
    """(cycles run, cycles replayed from their start) of a batch."""
    c, r = ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().md_batch_cycles(b, ctypes.byref(c), ctypes.byref(r)), "md_batch_cycles")
    return int(c.value), int(r.value)


def md_batch_cancel(b, ticket: int):
    _check(load().md_batch_cancel(b, ctypes.c_uint64(ticket)), "md_batch_cancel")


def md_batch_destroy(b):
    if b:
        _check(load().md_batch_destroy(b), "md_batch_destroy")


def md_atm_direct(pos, nu: float, precision: int = MD_FP32, stream=None):
    """All-triplet ATM forces (open boundaries, no cutoff): returns (f3 (n, 3), u3)."""
    n = int(np.asarray(pos).shape[0])
    x = _arr(pos, n)
    f = np.zeros((n, 3), dtype=np.float64)
    u = _D()
    _check(load().md_atm_direct(_ptr(x), n, float(nu), int(precision), _ptr(f), ctypes.byref(u),
                                stream if stream else None), "md_atm_direct")
    return f, u.value


def md_measure_fma_peak(kind: int, min_ms: float = 50.0):
    """FMA throughput of the device: kind 0 FP32, 1 packed FP32x2, 2 FP64.  Returns (flop/s, ms)."""
    f, ms = _D(), _D()
    _check(load().md_measure_fma_peak(int(kind), float(min_ms), ctypes.byref(f), ctypes.byref(ms)),
           "md_measure_fma_peak")
    return f.value, ms.value


def md_atm_forces_noalloc(d_pos_ptr: int, n: int, box_L: float, nu: float, rc_triplet: float, d_f3_ptr: int,
                          stream=None):
    """ATM forces without any device allocation: d_pos_ptr / d_f3_ptr are device addresses of
    n x 3 float64 arrays (caller order).  Returns (u3, triplets)."""
    u3 = _D()
    trip = ctypes.c_uint64()
    st = load().md_atm_forces_noalloc(ctypes.c_void_p(int(d_pos_ptr)), int(n), float(box_L), float(nu),
                                      float(rc_triplet), ctypes.c_void_p(int(d_f3_ptr)), ctypes.byref(u3),
                                      ctypes.byref(trip), None if stream is None else ctypes.c_void_p(int(stream)))
    _check(st, "md_atm_forces_noalloc")
    return u3.value, int(trip.value)


@dataclass
class System:
    """Owning handle around md_* calls (marshalling only)."""
    handle: object
    n: int
    L: float

    @classmethod
    def create(cls, pos, box_L, vel=None, mass=1.0, precision=MD_FP32, eps=1.0, sigma=1.0, rc_pair=2.5, nu=0.0,
               rc_triplet=2.5, skin=None, atm_kernel=-1, lj_kernel=-1):
        h = md_create_system(pos, box_L, vel, mass, precision)
        try:
            if skin is not None:
                md_set_skin(h, skin)
            md_set_potentials(h, eps, sigma, rc_pair, nu, rc_triplet)
            if atm_kernel != -1:
                md_set_atm_kernel(h, atm_kernel)
            if lj_kernel != -1:
                md_set_lj_kernel(h, lj_kernel)
        except Exception:
            md_destroy_system(h)
            raise
        return cls(h, int(np.asarray(pos).shape[0]), float(box_L))

    def step(self, n_outer, k_inner, dt_outer):
        md_respa_step(self.handle, n_outer, k_inner, dt_outer)

    def forces(self):
        return md_get_forces(self.handle)

    def energy(self):
        return md_get_energy(self.handle)

    def state(self):
        return md_get_state(self.handle)

    def set_distance_classes(self, r_a, s_near):
        md_set_distance_classes(self.handle, r_a, s_near)

    def near_forces(self):
        return md_get_near_forces(self.handle)

    def rdf(self, nbins, r_max):
        return md_get_rdf(self.handle, nbins, r_max)

    def set_state(self, pos=None, vel=None):
        md_set_state(self.handle, pos, vel)

    def stats(self):
        return md_get_stats(self.handle)

    def close(self):
        if self.handle:
            md_destroy_system(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
