"""CPU FP64 oracle for the r-RESPA LJ + ATM hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The GPU library neither imports nor links it,
and it imports nothing from the GPU library.

What it computes (arXiv 2507.11172):
  * ``lj_brute`` / ``lj_particles``   -- Lennard-Jones 12-6 forces, energy and
    virial over every unordered pair with r <= r_c (Sec. 2.1, Sec. 4.2.2).
  * ``atm_brute`` / ``atm_particles`` -- Axilrod-Teller-Muto forces, energy
    and virial over every unordered triple whose three pair distances are all
    <= r_c (Sec. 2.1; Fig. 2 caption; Sec. 4.2.2), literal cosine form.
  * ``respa.run``                     -- the single-loop r-RESPA integrator of
    Algorithm 2 (Sec. 4.1), written out step by step.

The force routines are plain C (``forces.c``, IEEE double, no FMA
contraction) compiled on first use with gcc; the integrator is numpy.
Pins: ``tests/test_oracle_*.py`` check closed forms, lattice sums,
finite-difference gradients, invariants and textbook special cases.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_lock = threading.Lock()
_lib = None

_D = ctypes.c_double
_I64 = ctypes.c_int64
_P = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile forces.c into oracle/_build/liboracle.so (idempotent)."""
    src = os.path.join(_HERE, "forces.c")
    out_dir = os.path.join(_HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, "liboracle.so")
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        tmp = so + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                               "-fno-fast-math", "-o", tmp, src, "-lm"])
        os.replace(tmp, so)
    return so


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.oracle_lj_brute.restype = ctypes.c_int
        lib.oracle_lj_brute.argtypes = [_I64, _P, _D, _D, _D, _D, _P, _P, _P]
        lib.oracle_lj_particles.restype = ctypes.c_int
        lib.oracle_lj_particles.argtypes = [_I64, _P, _D, _D, _D, _D, _I64, _P, _P, _P]
        lib.oracle_atm_brute.restype = ctypes.c_int
        lib.oracle_atm_brute.argtypes = [_I64, _P, _D, _D, _D, _P, _P, _P, _P]
        lib.oracle_atm_particles.restype = ctypes.c_int
        lib.oracle_atm_particles.argtypes = [_I64, _P, _D, _D, _D, _I64, _P, _P, _P, _P]
        lib.oracle_atm_triangle.restype = ctypes.c_int
        lib.oracle_atm_triangle.argtypes = [_P, _P, _P, _D, _P, _P]
        lib.oracle_kinetic.restype = ctypes.c_double
        lib.oracle_kinetic.argtypes = [_I64, _P, _D]
        _lib = lib
        return lib


def _pos(x) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    if x.ndim != 2 or x.shape[1] != 3:
        raise ValueError("positions must have shape (n, 3)")
    return x


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def lj_brute(x, L: float, eps: float = 1.0, sigma: float = 1.0, rc: float = 2.5):
    """Lennard-Jones over all unordered pairs: (F (n,3), U, W)."""
    x = _pos(x)
    n = x.shape[0]
    f = np.zeros((n, 3))
    u, w = _D(), _D()
    rc_ = _load().oracle_lj_brute(n, _ptr(x), L, eps, sigma, rc, _ptr(f), ctypes.byref(u), ctypes.byref(w))
    if rc_ != 0:
        raise ValueError("oracle_lj_brute: bad arguments")
    return f, u.value, w.value


def lj_particles(x, L: float, sel, eps: float = 1.0, sigma: float = 1.0, rc: float = 2.5):
    """Complete LJ force and pair-energy sum of the selected particles."""
    x = _pos(x)
    sel = np.ascontiguousarray(sel, dtype=np.int64)
    f = np.zeros((sel.size, 3))
    u = np.zeros(sel.size)
    rc_ = _load().oracle_lj_particles(x.shape[0], _ptr(x), L, eps, sigma, rc, sel.size, _ptr(sel), _ptr(f), _ptr(u))
    if rc_ != 0:
        raise ValueError("oracle_lj_particles: bad arguments")
    return f, u


def atm_brute(x, L: float, nu: float = 0.073, rc: float = 2.5):
    """ATM over all unordered triples: (F (n,3), U, W, n_triplets)."""
    x = _pos(x)
    n = x.shape[0]
    f = np.zeros((n, 3))
    u, w, c = _D(), _D(), _I64()
    rc_ = _load().oracle_atm_brute(n, _ptr(x), L, nu, rc, _ptr(f), ctypes.byref(u), ctypes.byref(w), ctypes.byref(c))
    if rc_ != 0:
        raise ValueError("oracle_atm_brute: bad arguments")
    return f, u.value, w.value, int(c.value)


def atm_particles(x, L: float, sel, nu: float = 0.073, rc: float = 2.5):
    """Complete ATM force, energy share and triplet count of the selected particles."""
    x = _pos(x)
    sel = np.ascontiguousarray(sel, dtype=np.int64)
    f = np.zeros((sel.size, 3))
    u = np.zeros(sel.size)
    c = np.zeros(sel.size, dtype=np.int64)
    rc_ = _load().oracle_atm_particles(x.shape[0], _ptr(x), L, nu, rc, sel.size, _ptr(sel), _ptr(f), _ptr(u), _ptr(c))
    if rc_ != 0:
        raise ValueError("oracle_atm_particles: bad arguments or neighbour overflow")
    return f, u, c


def atm_triangle(p, q, r, nu: float = 1.0):
    """phi3 of one explicit triangle and its gradients (rows: d/dp, d/dq, d/dr)."""
    p = np.ascontiguousarray(p, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    r = np.ascontiguousarray(r, dtype=np.float64)
    phi = _D()
    g = np.zeros((3, 3))
    _load().oracle_atm_triangle(_ptr(p), _ptr(q), _ptr(r), nu, ctypes.byref(phi), _ptr(g))
    return phi.value, g


def kinetic(v, m: float = 1.0) -> float:
    v = _pos(v)
    return float(_load().oracle_kinetic(v.shape[0], _ptr(v), m))


def wrap(x, L: float) -> np.ndarray:
    """Positions folded into [0, L) per axis (x - L floor(x / L))."""
    x = np.asarray(x, dtype=np.float64)
    return x - L * np.floor(x / L)
