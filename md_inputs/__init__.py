"""Seeded synthetic inputs for the r-RESPA three-body workloads.

This module is shared by the CPU oracle and the GPU path as a source of
*inputs only*: it holds none of the method's arithmetic (no potentials, no
forces, no integrator).  Every random number comes from a counter-based
splitmix64 stream (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), so a draw depends only on (seed, stream, counter)
and never on call order.

Workloads (reduced LJ units, m = 1, k_B = 1, as in the paper's Sec. 4.1):
  * ``fcc_jitter``  -- FCC lattice at density rho with seeded vacancies when N
    is not 4 n^3, Gaussian jitter per axis (the lattice-plus-jitter systems).
  * ``rsa``         -- random sequential addition with a minimum distance
    (liquid-like start).
  * ``maxwell``     -- Maxwell-Boltzmann velocities at temperature T with the
    centre-of-mass velocity removed and the kinetic temperature set exactly.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

SEED_BASE = 20250715

# stream identifiers: each kind of draw uses its own counter space
STREAM_VACANCY = 1
STREAM_JITTER = 2
STREAM_VELOCITY = 3
STREAM_RSA = 4
STREAM_ENSEMBLE = 5


def splitmix64(seed: int, stream: int, counters: np.ndarray) -> np.ndarray:
    """splitmix64 output for counter values ``counters`` of (seed, stream)."""
    c = np.asarray(counters, dtype=np.uint64)
    key = np.uint64((seed * 0x100000001B3 + stream * 0x9E3779B1) & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        z = key + (c + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, stream: int, start: int, n: int) -> np.ndarray:
    """n doubles in [0, 1) from counters start .. start+n-1 (53-bit mantissa)."""
    z = splitmix64(seed, stream, np.arange(start, start + n, dtype=np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def gaussian(seed: int, stream: int, start: int, n: int) -> np.ndarray:
    """n standard normal doubles by Box-Muller on pairs of uniforms."""
    m = (n + 1) // 2
    u = uniform(seed, stream, 2 * start, 2 * m)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    g = np.empty(2 * m)
    g[0::2] = r * np.cos(2.0 * np.pi * u2)
    g[1::2] = r * np.sin(2.0 * np.pi * u2)
    return g[:n]


def box_length(n: int, rho: float) -> float:
    return (n / rho) ** (1.0 / 3.0)


def fcc_jitter(n: int, rho: float, jitter: float, seed: int) -> tuple[np.ndarray, float]:
    """FCC positions (n, 3) in a periodic cube of side L = (n/rho)^(1/3).

    n_c = ceil((n/4)^(1/3)) cubic cells of edge L/n_c hold 4 n_c^3 sites; the
    4 n_c^3 - n sites with the largest seeded keys become vacancies, the rest
    keep their lattice order.  Each kept site gets N(0, jitter^2) per axis and
    is wrapped into [0, L).
    """
    L = box_length(n, rho)
    nc = int(math.ceil((n / 4.0) ** (1.0 / 3.0) - 1e-12))
    while 4 * nc ** 3 < n:
        nc += 1
    a = L / nc
    basis = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
    g = np.arange(nc)
    cz, cy, cx = np.meshgrid(g, g, g, indexing="ij")
    cells = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], axis=1).astype(np.float64)
    sites = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3) * a
    nsite = sites.shape[0]
    if nsite > n:
        keys = splitmix64(seed, STREAM_VACANCY, np.arange(nsite, dtype=np.uint64))
        keep = np.sort(np.argsort(keys, kind="stable")[:n])
        sites = sites[keep]
    x = sites + jitter * gaussian(seed, STREAM_JITTER, 0, 3 * n).reshape(n, 3)
    x = x - L * np.floor(x / L)
    x[x >= L] = 0.0
    return np.ascontiguousarray(x), L


def maxwell(n: int, temperature: float, seed: int, mass: float = 1.0) -> np.ndarray:
    """Velocities (n, 3): N(0, T/m) per component, zero total momentum, and
    sum(m v^2) / (3n - 3) == T exactly (up to rounding)."""
    v = gaussian(seed, STREAM_VELOCITY, 0, 3 * n).reshape(n, 3) * math.sqrt(temperature / mass)
    v -= v.mean(axis=0)
    t_now = mass * float(np.sum(v * v)) / (3 * n - 3)
    if t_now > 0:
        v *= math.sqrt(temperature / t_now)
    return np.ascontiguousarray(v)


_rsa_lock = threading.Lock()
_rsa_lib = None


def _load_rsa():
    global _rsa_lib
    with _rsa_lock:
        if _rsa_lib is not None:
            return _rsa_lib
        here = os.path.dirname(os.path.abspath(__file__))
        src = os.path.join(here, "rsa.c")
        out_dir = os.path.join(here, "_build")
        os.makedirs(out_dir, exist_ok=True)
        so = os.path.join(out_dir, "librsa.so")
        if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
            tmp = so + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, src, "-lm"])
            os.replace(tmp, so)
        lib = ctypes.CDLL(so)
        lib.rsa_place.restype = ctypes.c_int64
        lib.rsa_place.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                  ctypes.c_int64, ctypes.c_void_p]
        _rsa_lib = lib
        return lib


def rsa(n: int, rho: float, d_min: float, seed: int, max_trials_factor: int = 200) -> tuple[np.ndarray, float]:
    """Random sequential addition of n points in a periodic cube at density rho.

    Trial t draws a uniform point from counters 3t..3t+2 of (seed, STREAM_RSA)
    and is accepted iff it lies at least d_min (minimum image) from every point
    accepted before it.  Returns positions (n, 3) and L.
    """
    L = box_length(n, rho)
    lib = _load_rsa()
    out = np.zeros((n, 3), dtype=np.float64)
    got = lib.rsa_place(n, L, d_min, ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), n * max_trials_factor,
                        out.ctypes.data)
    if got != n:
        raise RuntimeError(f"RSA placed only {got} of {n} points (jamming?)")
    return out, L


@dataclass
class Workload:
    """One synthetic system: positions, velocities and the run parameters."""
    name: str
    x: np.ndarray
    v: np.ndarray
    L: float
    eps: float = 1.0
    sigma: float = 1.0
    rc2: float = 2.5
    nu: float = 0.073
    rc3: float = 2.5
    dt_outer: float = 0.01
    k_inner: int = 5
    n_outer: int = 10
    mass: float = 1.0
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


def config_seed(config: int, replica: int = 0) -> int:
    return SEED_BASE + 1000 * config + replica


def fcc_system(n: int, rho: float = 0.8, temperature: float = 1.0, jitter: float = 0.05, seed: int = 0,
               name: str = "fcc") -> Workload:
    x, L = fcc_jitter(n, rho, jitter, seed)
    v = maxwell(n, temperature, seed)
    return Workload(name=name, x=x, v=v, L=L)


def small_fcc_1k() -> Workload:
    """1,000 particles, FCC at density 0.8, jitter 0.05 sigma, T*=1.0; LJ
    eps=sigma=1, r_c=2.5; ATM nu=0.073, r_c=2.5; dt_outer=0.01, k=5, 10 outer."""
    w = fcc_system(1000, 0.8, 1.0, 0.05, config_seed(1), name="fcc1k_rho0.8")
    w.dt_outer, w.k_inner, w.n_outer = 0.01, 5, 10
    return w


def fcc_100k(replica: int = 0) -> Workload:
    """100,000 particles, same lattice/jitter/potentials, k=10, dt_outer=0.02,
    100 outer steps.  `replica` selects an independent seed (one per rank when
    several GPUs each run their own copy)."""
    w = fcc_system(100_000, 0.8, 1.0, 0.05, config_seed(2, replica), name="fcc100k_rho0.8")
    w.dt_outer, w.k_inner, w.n_outer = 0.02, 10, 100
    return w


def rsa_2m(rc3: float = 2.5, n: int = 2_000_000) -> Workload:
    """2,000,000 particles, RSA start (d_min 0.9) at density 0.75, T*=1.2,
    triplet cutoff 2.0 or 2.5, k=10, dt_outer=0.02, 50 outer steps."""
    seed = config_seed(3)
    x, L = rsa(n, 0.75, 0.9, seed)
    v = maxwell(n, 1.2, seed)
    w = Workload(name=f"rsa2m_rho0.75_rc3_{rc3}", x=x, v=v, L=L, rc3=rc3)
    w.dt_outer, w.k_inner, w.n_outer = 0.02, 10, 50
    return w


def ensemble_specs(n_replicas: int = 256, seed: int | None = None, n_lo: int = 500, n_hi: int = 20000):
    """Per-replica (n, rho, T, k) for the batched ensemble: n log-uniform in
    [n_lo, n_hi], rho ~ U[0.6, 0.9], T ~ U[0.8, 1.5], k in {4, 8, 16}."""
    seed = config_seed(4) if seed is None else seed
    u = uniform(seed, STREAM_ENSEMBLE, 0, 4 * n_replicas).reshape(n_replicas, 4)
    n = np.exp(np.log(n_lo) + u[:, 0] * (np.log(n_hi) - np.log(n_lo))).astype(np.int64)
    rho = 0.6 + 0.3 * u[:, 1]
    temp = 0.8 + 0.7 * u[:, 2]
    k = np.array([4, 8, 16])[np.minimum((u[:, 3] * 3).astype(np.int64), 2)]
    return [dict(n=int(n[i]), rho=float(rho[i]), T=float(temp[i]), k=int(k[i])) for i in range(n_replicas)]


def ensemble_replica(spec: dict, replica: int, seed_config: int = 4, dt_inner: float = 0.002) -> Workload:
    seed = config_seed(seed_config, replica + 1)
    w = fcc_system(spec["n"], spec["rho"], spec["T"], 0.05, seed, name=f"replica{replica}")
    w.k_inner = spec["k"]
    w.dt_outer = spec["k"] * dt_inner
    w.n_outer = spec.get("n_outer", 20)
    return w
