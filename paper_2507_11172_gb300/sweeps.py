"""Energy-conservation sweep of the method (Sec. 4.2.1, toy scenario): relative variation in true
energy, RVITE (Eq. 4), over the step-size factor s and the ATM strength nu, and the histogram of the
relative deviation of the total energy from the Stormer-Verlet run (s = 1) at the same times.

Scenario (Sec. 4.2): 675 particles in a periodic 10 x 10 x 10 box, eps = sigma = m = 1,
dt = 0.001 (the paper's inner step), 24 000 iterations, s = 1 .. 12, nu in [0.05, 1.0].  The paper
does not state the cutoff or the initial state: this sweep uses r_c2 = r_c3 = 2.5, an FCC lattice with
0.05 sigma jitter and Maxwell velocities at T* = 1.0, equilibrated for 2 000 Stormer-Verlet
iterations (s = 1) before the measured run.  The total energy e(i) = E_kin + U2 + U3 is read at
every full step (iterations divisible by s; Sec. 4.1) and RVITE = mean_i |e(i) - mean(e)| / mean(E_kin).

Aluminium scenario (--scenario aluminium; Sec. 4.3, Table 1): 4995 particles in a 20 x 20 x 20 box,
dt = 0.00304, nu = 0.3095, T* = 1.1, 24 000 iterations.  The paper runs it with open boundaries and
states no cutoff; here it is periodic with r_c2 = r_c3 = 2.5 and starts from the same kind of jittered
FCC state (no equilibrated aluminium configuration is available).

Everything runs through the C ABI (md_respa_step with k_inner = s, dt_outer = s dt; md_get_energy).

    python -m paper_2507_11172_gb300.sweeps [--scenario toy|aluminium] [--iters 24000]
        [--nus 0.05,0.25,0.5,0.75,1.0] [--s 1,2,...]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import MD_FP32, MD_FP64, System


def toy_state(n: int = 675, L: float = 10.0, temperature: float = 1.0, seed: int = 2507):
    """FCC sites of the box (4 nc^3 >= n, seeded vacancies), 0.05 sigma jitter, Maxwell velocities."""
    import md_inputs
    x, Lx = md_inputs.fcc_jitter(n, n / L ** 3, 0.05, seed)
    v = md_inputs.maxwell(n, temperature, seed + 1)
    return x, Lx, v


# (n, box side, T*, dt, default nu values) of the two scenarios of Sec. 4.2-4.3
SCENARIOS = {
    "toy": (675, 10.0, 1.0, 0.001, "0.05,0.25,0.5,0.75,1.0"),
    "aluminium": (4995, 20.0, 1.1, 0.00304, "0.3095"),
}


def rvite(e_tot, e_kin) -> float:
    """Eq. 4: (1 / (K J)) sum_i |e(i) - mean(e)|, K the mean kinetic energy, J the number of full steps."""
    e_tot = np.asarray(e_tot, dtype=np.float64)
    return float(np.mean(np.abs(e_tot - e_tot.mean())) / np.mean(e_kin))


def deviation_histogram(e_s, e_1, s: int, bins: int = 50):
    """Sec. 4.2.1: relative deviation of the total energy of a run with step-size factor s from the
    Stormer-Verlet run (s = 1) at the same times, (E_s(j) - E_1(j s)) / |E_1(j s)|, as a histogram of
    `bins` equal bins over its range.  e_s[j] is the energy after j + 1 full steps of s iterations,
    e_1[k] after k + 1 iterations.  Returns (counts, edges)."""
    e_1 = np.asarray(e_1, dtype=np.float64)[s - 1::s]
    e_s = np.asarray(e_s, dtype=np.float64)
    m = min(len(e_1), len(e_s))
    dev = (e_s[:m] - e_1[:m]) / np.abs(e_1[:m])
    return np.histogram(dev, bins=bins)


def run_point(x, L, v, nu: float, s: int, iters: int, dt: float = 0.001, equil: int = 2000,
              precision: int = MD_FP32, rc: float = 2.5):
    """One (nu, s) point: returns (RVITE, energies (J, 3) = (E_kin, U2, U3) at the full steps, seconds)."""
    with System.create(x, L, v, precision=precision, nu=nu, rc_pair=rc, rc_triplet=rc) as sysm:
        for _ in range(equil // 100):  # equilibration in calls of 100 Stormer-Verlet iterations
            sysm.step(100, 1, dt)
        e = []
        t0 = time.perf_counter()
        for _ in range(iters // s):
            sysm.step(1, s, s * dt)
            ek, u2, u3, _ = sysm.energy()
            e.append((ek, u2, u3))
        dt_wall = time.perf_counter() - t0
    e = np.asarray(e)
    return rvite(e.sum(1), e[:, 0]), e, dt_wall


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--scenario", default="toy", choices=sorted(SCENARIOS))
    ap.add_argument("--iters", type=int, default=24000)
    ap.add_argument("--nus", default=None)
    ap.add_argument("--s", default=",".join(str(k) for k in range(1, 13)))
    ap.add_argument("--fp64", action="store_true")
    args = ap.parse_args(argv)
    n, box, temp, dt, nus = SCENARIOS[args.scenario]
    x, L, v = toy_state(n, box, temp)
    out = []
    for nu in [float(a) for a in (args.nus or nus).split(",")]:
        e_sv = None  # the Stormer-Verlet (s = 1) energies of this nu, for the deviation histogram
        for s in [int(a) for a in args.s.split(",")]:
            r, e, wall = run_point(x, L, v, nu, s, args.iters, dt=dt, precision=MD_FP64 if args.fp64 else MD_FP32)
            point = {"scenario": args.scenario, "nu": nu, "s": s, "rvite": r, "full_steps": len(e), "seconds": wall,
                     "e_mean": float(e.sum(1).mean()),
                     "max_dev_rel": float(np.abs(e.sum(1) - e.sum(1).mean()).max() / abs(e.sum(1).mean()))}
            if s == 1:
                e_sv = e.sum(1)
            elif e_sv is not None:
                counts, edges = deviation_histogram(e.sum(1), e_sv, s)
                point["dev_hist"] = {"lo": float(edges[0]), "hi": float(edges[-1]), "counts": counts.tolist()}
            out.append(point)
            print(json.dumps(out[-1]), flush=True)
    return out


if __name__ == "__main__":
    main()
