"""Linked-cell CPU baseline (FP64, OpenMP) of the method's forces and its r-RESPA integrator.

The CPU throughput figure the GPU path is compared with (the paper's shared-memory Cutoff traversal:
linked cells, every particle against its 27 surrounding cells, no Newton 3).  It is measurement
infrastructure, not the parity oracle and not the product: ``tests/test_cpu_cells.py`` pins it against
the brute-force oracle, ``bench.py`` times it, and it shares no code with ``oracle/`` or with the CUDA
library.  ``cells.c`` is compiled with gcc on first use (``-O3 -fopenmp``, no FMA contraction); the
thread count is OpenMP's (``OMP_NUM_THREADS``, else every host core).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_lock = threading.Lock()
_lib = None
_D, _I, _I64, _P = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile cells.c into cpu_cells/_build/libcpucells.so (idempotent)."""
    src = os.path.join(_HERE, "cells.c")
    out_dir = os.path.join(_HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, "libcpucells.so")
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        tmp = so + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O3", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, so)
    return so


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.cells_forces.restype = _I
            lib.cells_forces.argtypes = [_I64, _P, _D, _D, _D, _D, _D, _D, _P, _P, _P]
            lib.cells_respa.restype = _I
            lib.cells_respa.argtypes = [_I64, _P, _P, _D, _D, _D, _D, _D, _D, _D, _I, _I, _D, _P, _P, _I, _P]
            lib.cells_threads.restype = _I
            lib.cells_threads.argtypes = []
            _lib = lib
        return _lib


def _arr(x) -> np.ndarray:
    a = np.array(x, dtype=np.float64, order="C", copy=True)
    if a.ndim != 2 or a.shape[1] != 3:
        raise ValueError("arrays must have shape (n, 3)")
    return a


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(st: int, what: str):
    if st == -1:
        raise ValueError(f"{what}: bad arguments or a box of fewer than three cells per side of the largest cutoff")
    if st != 0:
        raise MemoryError(f"{what}: out of host memory")


def threads() -> int:
    """OpenMP threads the baseline runs on."""
    return int(_load().cells_threads())


def forces(x, L: float, eps: float = 1.0, sigma: float = 1.0, rc2: float = 2.5, nu: float = 0.073, rc3: float = 2.5):
    """F2 (n, 3), F3 (n, 3) and a dict with U2, W2, U3 and the number of triplets within r_c3."""
    x = _arr(x)
    n = x.shape[0]
    f2, f3, out = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(4)
    _check(_load().cells_forces(n, _p(x), L, eps, sigma, rc2, nu, rc3, _p(f2), _p(f3), _p(out)), "cells_forces")
    return f2, f3, {"u2": float(out[0]), "w2": float(out[1]), "u3": float(out[2]), "triplets": int(out[3])}


class State:
    """Positions, velocities and the forces at those positions, advanced in place by ``run``."""

    def __init__(self, x, v, L: float, mass: float = 1.0, eps: float = 1.0, sigma: float = 1.0, rc2: float = 2.5,
                 nu: float = 0.073, rc3: float = 2.5):
        self.x, self.v = _arr(x), _arr(v)
        if self.x.shape != self.v.shape:
            raise ValueError("x and v must have the same shape")
        self.L, self.mass, self.eps, self.sigma, self.rc2, self.nu, self.rc3 = L, mass, eps, sigma, rc2, nu, rc3
        self.f2, self.f3 = np.zeros_like(self.x), np.zeros_like(self.x)
        self.have_forces = False

    def run(self, n_outer: int, k_inner: int, dt_outer: float) -> dict:
        """Algorithm 2 for n_outer outer steps of k_inner inner steps; returns U2 and U3 at the end, the
        interacting triplets summed over the ATM evaluations, and the seconds spent in the LJ and ATM
        evaluations and in the whole call."""
        out = np.zeros(6)
        t0 = time.perf_counter()
        st = _load().cells_respa(self.x.shape[0], _p(self.x), _p(self.v), self.L, self.mass, self.eps, self.sigma,
                                 self.rc2, self.nu, self.rc3, int(n_outer), int(k_inner), float(dt_outer),
                                 _p(self.f2), _p(self.f3), 1 if self.have_forces else 0, _p(out))
        secs = time.perf_counter() - t0
        _check(st, "cells_respa")
        self.have_forces = True
        return {"u2": float(out[0]), "u3": float(out[1]), "triplets": float(out[2]), "lj_s": float(out[3]),
                "atm_s": float(out[4]), "atm_evals": int(out[5]), "seconds": secs}
