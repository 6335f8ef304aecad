"""Single-loop r-RESPA integrator (Algorithm 2, Sec. 4.1) -- oracle, test use only.

The two force fields are split as in the paper: the Lennard-Jones pair force
F2b is integrated every iteration of step dt, the ATM triplet force F3b only
with the step-size factor s (a kick of dt*s/(2m) on iterations with i % s == 0
and after iterations with (i+1) % s == 0).  With s = 1 this is Stormer-Verlet
(Sec. 4.1, "Performance" item).  Only iterations divisible by s are full steps
where energies are meaningful.

Readings where the paper leaves a choice:
  * the public call takes the outer step dt_outer and k = s inner steps, so the
    paper's dt is dt_outer / k;
  * positions are folded back into the periodic box after every position
    update (Cutoff runs use periodic boundaries, Sec. 4.2);
  * F2b and F3b are cached between calls: Algorithm 2 evaluates them at x^0
    once, before its loop.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np

from . import atm_brute, kinetic, lj_brute, wrap

ForceFn = Callable[[np.ndarray], tuple]  # x -> (F, U, W)


@dataclass
class State:
    x: np.ndarray
    v: np.ndarray
    L: float
    mass: float = 1.0
    f2: Optional[np.ndarray] = None
    f3: Optional[np.ndarray] = None
    u2: float = 0.0
    u3: float = 0.0
    w2: float = 0.0
    w3: float = 0.0
    energies: list = field(default_factory=list)  # (e_kin, u2, u3) at each full step


def lj_atm_forces(L: float, eps: float, sigma: float, rc2: float, nu: float, rc3: float):
    """The two brute-force force fields of the method as callables x -> (F, U, W)."""
    def f2(x):
        return lj_brute(x, L, eps, sigma, rc2)

    def f3(x):
        f, u, w, _ = atm_brute(x, L, nu, rc3)
        return f, u, w
    return f2, f3


def run(state: State, n_outer: int, k_inner: int, dt_outer: float, f2b: ForceFn, f3b: ForceFn,
        periodic: bool = True, record: bool = False) -> State:
    """Advance ``state`` by n_outer outer steps of k_inner inner steps (Algorithm 2, s = k_inner,
    dt = dt_outer / k_inner).  Updates the state in place and returns it."""
    if n_outer < 0 or k_inner < 1 or not dt_outer > 0:
        raise ValueError("n_outer >= 0, k_inner >= 1 and dt_outer > 0 required")
    s = k_inner
    dt = dt_outer / k_inner
    m = state.mass
    x, v = state.x, state.v
    if state.f2 is None:  # calculate F2b(x^0)
        state.f2, state.u2, state.w2 = f2b(x)
    if state.f3 is None:  # calculate F3b(x^0)
        state.f3, state.u3, state.w3 = f3b(x)
    f2, f3 = state.f2, state.f3
    for i in range(n_outer * s):
        is_respa = (i % s) == 0
        next_is_respa = ((i + 1) % s) == 0
        if is_respa:
            v = v + (dt * s / (2.0 * m)) * f3
        x_new = x + dt * v + (dt * dt / (2.0 * m)) * f2
        if periodic:
            x_new = wrap(x_new, state.L)
        f2_new, state.u2, state.w2 = f2b(x_new)
        v = v + (dt / (2.0 * m)) * (f2 + f2_new)
        x, f2 = x_new, f2_new
        if next_is_respa:
            f3, state.u3, state.w3 = f3b(x)
            v = v + (dt * s / (2.0 * m)) * f3
            if record:
                state.energies.append((kinetic(v, m), state.u2, state.u3))
    state.x, state.v, state.f2, state.f3 = x, v, f2, f3
    return state


def rvite(e_tot: np.ndarray, e_kin: np.ndarray) -> float:
    """Relative variation in true energy (Eq. 4): mean |e(i) - mean(e)| / mean(K)."""
    e_tot = np.asarray(e_tot, dtype=np.float64)
    return float(np.mean(np.abs(e_tot - e_tot.mean())) / np.mean(e_kin))


# ---------------------------------------------------------------------------------------------
# Distance classes for the three-body force (the outlook of Sec. 5, after Nakano et al. and
# Grubmueller et al., Sec. 3): an intermediate triplet cutoff r_a < r_c splits the ATM triplets
# into a near class (all three pair distances <= r_a) and a far class (the other triplets with all
# three distances <= r_c).  r-RESPA with three levels (Sec. 2.3.1: "an arbitrary number of
# separations ... nested loop"): the LJ force every iteration of step dt, the near triplets with the
# step-size factor s_near (every s_near iterations), the far triplets with s = k_inner.

@dataclass
class State3:
    x: np.ndarray
    v: np.ndarray
    L: float
    mass: float = 1.0
    f2: Optional[np.ndarray] = None
    f3n: Optional[np.ndarray] = None
    f3f: Optional[np.ndarray] = None
    u2: float = 0.0
    u3n: float = 0.0
    u3f: float = 0.0
    energies: list = field(default_factory=list)  # (e_kin, u2, u3n + u3f) at each full step


def class_forces(L: float, nu: float, r_a: float, rc3: float):
    """Near and far ATM force fields x -> (F, U, W): near = every triplet within r_a (the triplet
    cutoff r_a), far = the triplets within r_c minus the near ones."""
    def near(x):
        f, u, w, _ = atm_brute(x, L, nu, r_a)
        return f, u, w

    def far(x):
        fa, ua, wa, _ = atm_brute(x, L, nu, rc3)
        fn, un, wn, _ = atm_brute(x, L, nu, r_a)
        return fa - fn, ua - un, wa - wn
    return near, far


def run3(state: State3, n_outer: int, k_inner: int, s_near: int, dt_outer: float, f2b: ForceFn,
         f3near: ForceFn, f3far: ForceFn, periodic: bool = True, record: bool = False) -> State3:
    """n_outer outer steps of k_inner iterations (dt = dt_outer / k_inner), written as one loop in
    the manner of Algorithm 2: the far kick dt k_inner / (2m) F3far opens and closes every block of
    k_inner iterations, the near kick dt s_near / (2m) F3near every block of s_near iterations, and
    every iteration is a velocity-Verlet step with F2.  s_near must divide k_inner."""
    if n_outer < 0 or k_inner < 1 or s_near < 1 or k_inner % s_near or not dt_outer > 0:
        raise ValueError("n_outer >= 0, s_near | k_inner and dt_outer > 0 required")
    dt = dt_outer / k_inner
    m = state.mass
    x, v = state.x, state.v
    if state.f2 is None:
        state.f2, state.u2, _ = f2b(x)
    if state.f3n is None:
        state.f3n, state.u3n, _ = f3near(x)
    if state.f3f is None:
        state.f3f, state.u3f, _ = f3far(x)
    f2, f3n, f3f = state.f2, state.f3n, state.f3f
    for i in range(n_outer * k_inner):
        if i % k_inner == 0:
            v = v + (dt * k_inner / (2.0 * m)) * f3f
        if i % s_near == 0:
            v = v + (dt * s_near / (2.0 * m)) * f3n
        x_new = x + dt * v + (dt * dt / (2.0 * m)) * f2
        if periodic:
            x_new = wrap(x_new, state.L)
        f2_new, state.u2, _ = f2b(x_new)
        v = v + (dt / (2.0 * m)) * (f2 + f2_new)
        x, f2 = x_new, f2_new
        if (i + 1) % s_near == 0:
            f3n, state.u3n, _ = f3near(x)
            v = v + (dt * s_near / (2.0 * m)) * f3n
        if (i + 1) % k_inner == 0:
            f3f, state.u3f, _ = f3far(x)
            v = v + (dt * k_inner / (2.0 * m)) * f3f
            if record:
                state.energies.append((kinetic(v, m), state.u2, state.u3n + state.u3f))
    state.x, state.v, state.f2, state.f3n, state.f3f = x, v, f2, f3n, f3f
    return state


# ---------------------------------------------------------------------------------------------
# Several distance classes (the outlook of Sec. 5 names several intermediate cutoffs, each class with
# its own time step): cutoffs r_1 < r_2 < ... < r_C = r_c3 split the ATM triplets by their largest pair
# distance, class c holding the triplets with r_{c-1} < max distance <= r_c (r_0 = 0).  Class c is
# integrated with step-size factor s_c, s_1 | s_2 | ... | s_C = k_inner, written as one loop in the
# manner of Algorithm 2: the class-c kicks dt s_c / (2m) F_c open and close every block of s_c
# iterations, the LJ force drives every iteration.

@dataclass
class StateN:
    x: np.ndarray
    v: np.ndarray
    L: float
    mass: float = 1.0
    f2: Optional[np.ndarray] = None
    f3: Optional[list] = None          # per-class forces
    u2: float = 0.0
    u3: Optional[list] = None          # per-class energies
    energies: list = field(default_factory=list)  # (e_kin, u2, sum of class energies) at each full step


def band_forces(L: float, nu: float, cutoffs):
    """Force fields x -> (F, U, W) of the classes r_{c-1} < max pair distance <= r_c, each the difference
    of two brute-force sums with the triplet cutoffs r_c and r_{c-1}."""
    cut = [float(c) for c in cutoffs]
    if any(not (b > a) for a, b in zip(cut, cut[1:])) or not cut[0] > 0:
        raise ValueError("cutoffs must increase from a positive value")

    def make(c):
        def f(x):
            fa, ua, wa, _ = atm_brute(x, L, nu, cut[c])
            if c == 0:
                return fa, ua, wa
            fb, ub, wb, _ = atm_brute(x, L, nu, cut[c - 1])
            return fa - fb, ua - ub, wa - wb
        return f
    return [make(c) for c in range(len(cut))]


def run_classes(state: StateN, n_outer: int, k_inner: int, s_list, dt_outer: float, f2b: ForceFn, fclass,
                periodic: bool = True, record: bool = False) -> StateN:
    """n_outer outer steps of k_inner iterations (dt = dt_outer / k_inner) with the classes' force fields
    fclass[c] kicked every s_list[c] iterations; s_list increasing, each dividing the next, the last
    equal to k_inner.  With two classes this is run3."""
    s_list = [int(s) for s in s_list]
    if (len(s_list) != len(fclass) or s_list[-1] != k_inner or any(s < 1 for s in s_list)
            or any(b % a for a, b in zip(s_list, s_list[1:])) or n_outer < 0 or not dt_outer > 0):
        raise ValueError("s_1 | s_2 | ... | s_C = k_inner, one factor per class, dt_outer > 0 required")
    dt = dt_outer / k_inner
    m = state.mass
    C = len(s_list)
    x, v = state.x, state.v
    if state.f2 is None:
        state.f2, state.u2, _ = f2b(x)
    if state.f3 is None:
        res = [f(x) for f in fclass]
        state.f3, state.u3 = [r[0] for r in res], [r[1] for r in res]
    f2, f3 = state.f2, list(state.f3)
    for i in range(n_outer * k_inner):
        for c in reversed(range(C)):  # opening kicks, slowest class first
            if i % s_list[c] == 0:
                v = v + (dt * s_list[c] / (2.0 * m)) * f3[c]
        x_new = x + dt * v + (dt * dt / (2.0 * m)) * f2
        if periodic:
            x_new = wrap(x_new, state.L)
        f2_new, state.u2, _ = f2b(x_new)
        v = v + (dt / (2.0 * m)) * (f2 + f2_new)
        x, f2 = x_new, f2_new
        for c in range(C):  # closing kicks, fastest class first
            if (i + 1) % s_list[c] == 0:
                f3[c], state.u3[c], _ = fclass[c](x)
                v = v + (dt * s_list[c] / (2.0 * m)) * f3[c]
        if (i + 1) % k_inner == 0 and record:
            state.energies.append((kinetic(v, m), state.u2, float(sum(state.u3))))
    state.x, state.v, state.f2, state.f3 = x, v, f2, f3
    return state
