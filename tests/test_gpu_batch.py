"""Batched ensemble and continuous serving: every request's result must equal the same request
run alone (md_respa_step), within the FP tolerances of the single-system tests, whatever else
shares the launches; the FP64 batch must also follow Algorithm 2 of the oracle."""
import numpy as np
import pytest

import md_inputs
import oracle
from oracle import respa

pytestmark = pytest.mark.gpu

NU = 0.073


def _systems(seed0=11):
    """Uneven replicas: sizes, densities, temperatures and step-size factors differ."""
    specs = [(600, 0.8, 1.0, 4), (1100, 0.85, 1.2, 8), (700, 0.7, 0.9, 2), (900, 0.75, 1.4, 1), (1500, 0.8, 1.1, 4)]
    out = []
    for i, (n, rho, T, k) in enumerate(specs):
        w = md_inputs.fcc_system(n, rho, T, 0.05, seed0 + i)
        w.k_inner = k
        w.dt_outer = 0.002 * k
        out.append(w)
    return out


def _alone(r3, w, n_outer, prec):
    with r3.System.create(w.x, w.L, w.v, precision=prec, nu=NU) as s:
        s.step(n_outer, w.k_inner, w.dt_outer)
        x, v = s.state()
        e = s.energy()
    return x, v, e


def _dist(a, b, L):
    d = a - b
    d -= L * np.rint(d / L)
    return np.abs(d).max()


@pytest.mark.parametrize("prec", [0, 1])
def test_each_result_same_alone_and_in_the_mix(gpu_lib, prec):
    r3 = gpu_lib
    ws = _systems()
    n_outer = 5
    alone = [_alone(r3, w, n_outer, prec) for w in ws]
    b = r3.md_batch_create(0)
    hs, tickets = [], []
    try:
        for w in ws:
            h = r3.md_create_system(w.x, w.L, w.v, 1.0, prec)
            r3.md_set_potentials(h, 1.0, 1.0, 2.5, NU, 2.5)
            hs.append(h)
            tickets.append(r3.md_batch_submit(b, h, n_outer, w.k_inner, w.dt_outer))
        r3.md_batch_run(b, 0)
        xtol = 1e-6 if prec == 0 else 1e-11
        for w, h, t, (xa, va, ea) in zip(ws, hs, tickets, alone):
            assert r3.md_batch_poll(b, t)
            x, v = r3.md_get_state(h)
            e = r3.md_get_energy(h)
            assert _dist(x, xa, w.L) < xtol
            assert np.abs(v - va).max() < 10 * xtol
            scale = abs(ea[0]) + abs(ea[1]) + abs(ea[2])
            assert abs(sum(e[:3]) - sum(ea[:3])) / scale < (1e-6 if prec == 0 else 1e-11)
            lat = r3.md_batch_latency(b, t)
            assert lat.size == n_outer and np.all(lat > 0)
    finally:
        r3.md_batch_destroy(b)
        for h in hs:
            r3.md_destroy_system(h)


def test_batch_fp64_follows_algorithm2(gpu_lib):
    r3 = gpu_lib
    ws = _systems(31)[:3]
    b = r3.md_batch_create(0)
    hs = []
    try:
        tickets = []
        for w in ws:
            h = r3.md_create_system(w.x, w.L, w.v, 1.0, r3.MD_FP64)
            r3.md_set_potentials(h, 1.0, 1.0, 2.5, NU, 2.5)
            hs.append(h)
            tickets.append(r3.md_batch_submit(b, h, 3, w.k_inner, w.dt_outer))
        r3.md_batch_run(b, 0)
        assert all(r3.md_batch_poll(b, t) for t in tickets)
        for w, h in zip(ws, hs):
            st = respa.State(w.x.copy(), w.v.copy(), w.L)
            f2b, f3b = respa.lj_atm_forces(w.L, 1.0, 1.0, 2.5, NU, 2.5)
            respa.run(st, 3, w.k_inner, w.dt_outer, f2b, f3b)
            x, v = r3.md_get_state(h)
            assert _dist(x, st.x, w.L) < 1e-10
            assert np.abs(v - st.v).max() < 1e-9
    finally:
        r3.md_batch_destroy(b)
        for h in hs:
            r3.md_destroy_system(h)


def test_serving_budget_and_arrivals(gpu_lib):
    """Deferred systems admitted by a memory budget that holds about two at a time; more
    requests arrive while others run; all finish and equal their lone runs."""
    r3 = gpu_lib
    ws = _systems(51)
    n_outer = 4
    alone = [_alone(r3, w, n_outer, 0) for w in ws]
    hs = []
    for w in ws:
        h = r3.md_create_system(w.x, w.L, w.v, 1.0, r3.MD_FP32 | r3.MD_DEFERRED)
        r3.md_set_potentials(h, 1.0, 1.0, 2.5, NU, 2.5)
        hs.append(h)
    # budget: about two of the largest systems
    b = r3.md_batch_create(2 * 400 * 1024 * 1024 // 100)
    try:
        tickets = [r3.md_batch_submit(b, hs[0], n_outer, ws[0].k_inner, ws[0].dt_outer),
                   r3.md_batch_submit(b, hs[1], n_outer, ws[1].k_inner, ws[1].dt_outer)]
        r3.md_batch_run(b, 8)  # a partial run, then more arrivals
        for w, h in zip(ws[2:], hs[2:]):
            tickets.append(r3.md_batch_submit(b, h, n_outer, w.k_inner, w.dt_outer))
        q, res = r3.md_batch_pending(b)
        assert q + res >= 3
        r3.md_batch_run(b, 0)
        for w, h, t, (xa, va, _) in zip(ws, hs, tickets, alone):
            assert r3.md_batch_poll(b, t)
            x, _ = r3.md_get_state(h)
            assert _dist(x, xa, w.L) < 1e-6
    finally:
        r3.md_batch_destroy(b)
        for h in hs:
            r3.md_destroy_system(h)


@pytest.mark.parametrize("prec", [0, 1])
def test_skin_violations_in_the_mix(gpu_lib, prec):
    """A thin skin (0.02) makes particles leave it within a cycle: the batch replays and then runs
    safe cycles (binning before any tick whose positions moved more than skin / 2); every result still
    equals the same request run alone (FP64: and follows Algorithm 2)."""
    r3 = gpu_lib
    ws = _systems(71)
    n_outer = 6
    alone = []
    for w in ws:
        with r3.System.create(w.x, w.L, w.v, precision=prec, nu=NU, skin=0.02) as s:
            s.step(n_outer, w.k_inner, w.dt_outer)
            alone.append(s.state())
    b = r3.md_batch_create(0)
    hs, tickets = [], []
    try:
        for w in ws:
            h = r3.md_create_system(w.x, w.L, w.v, 1.0, prec)
            r3.md_set_skin(h, 0.02)
            r3.md_set_potentials(h, 1.0, 1.0, 2.5, NU, 2.5)
            hs.append(h)
            tickets.append(r3.md_batch_submit(b, h, n_outer, w.k_inner, w.dt_outer))
        r3.md_batch_run(b, 0)
        cycles, replayed = r3.md_batch_cycles(b)
        assert replayed >= 1
        xtol = 1e-6 if prec == 0 else 1e-11
        for w, h, t, (xa, va) in zip(ws, hs, tickets, alone):
            assert r3.md_batch_poll(b, t)
            x, v = r3.md_get_state(h)
            assert _dist(x, xa, w.L) < xtol
            assert np.abs(v - va).max() < 10 * xtol
    finally:
        r3.md_batch_destroy(b)
        for h in hs:
            r3.md_destroy_system(h)


def _oracle_at(w, x, v):
    """LJ and ATM forces and energies of the oracle (per-particle pass over every particle) at the
    positions x the GPU produced, and the kinetic energy of v."""
    allp = np.arange(x.shape[0])
    f2, u2 = oracle.lj_particles(x, w.L, allp, 1.0, 1.0, 2.5)
    f3, u3, _ = oracle.atm_particles(x, w.L, allp, NU, 2.5)
    return f2, f3, oracle.kinetic(v), u2.sum() / 2, u3.sum() / 3


def _force_err(got, ref):
    frms = np.sqrt((ref ** 2).sum(1).mean())
    return float((np.linalg.norm(got - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), frms)).max())


def _served_mix(seed0):
    """Five small uneven replicas (3 outer steps each) and one of 24,000 particles (rotation kernel,
    large-N capacities; k = 10 at dt_outer = 0.02, 6 outer steps, so it stays resident over two cycles)."""
    ws = _systems(seed0)
    for w in ws:
        w.n_outer = 3
    big = md_inputs.fcc_system(24000, 0.8, 1.0, 0.05, seed0 + 99)
    big.k_inner = 10
    big.dt_outer = 0.02
    big.n_outer = 6
    return ws[:2] + [big] + ws[2:]


def test_served_fp32_matches_the_oracle_and_equals_alone_bitwise(gpu_lib):
    """Serving with deferred systems, a memory budget that holds the 24,000-particle member and only
    part of the small ones, and requests arriving while cycles run, FP32 forces with the rotation
    triplet kernel:
      * a request that does not fit waits in the queue while others are resident;
      * every request's cached forces at its final positions equal the oracle's at those positions
        (per-particle relative error <= 1e-5, every particle), and its energies (E_kin, U2, U3) agree
        within 1e-6 of E_kin + |U2| + |U3|;
      * every request's final state and forces equal the same request run alone bit for bit (the
        triplet forces are summed in fixed point, so the order in which launches mix does not matter;
        batches use the row LJ kernel, so the lone run uses it too)."""
    r3 = gpu_lib
    ws = _served_mix(131)
    alone = []
    for w in ws:
        with r3.System.create(w.x, w.L, w.v, precision=0, nu=NU, atm_kernel=2, lj_kernel=0) as s:
            s.step(w.n_outer, w.k_inner, w.dt_outer)
            alone.append((*s.state(), *s.forces()))
    hs = []
    for w in ws:
        h = r3.md_create_system(w.x, w.L, w.v, 1.0, r3.MD_FP32 | r3.MD_DEFERRED)
        r3.md_set_potentials(h, 1.0, 1.0, 2.5, NU, 2.5)
        r3.md_set_atm_kernel(h, 2)
        hs.append(h)
    need = [r3.md_get_memory(h) for h in hs]
    # the large member, the first two small ones, and then room for the smaller of the late ones only
    budget = need[2] + max(need[0] + need[1], need[3] + 0.5 * min(need[4], need[5]))
    assert need[2] + need[3] + need[4] + need[5] > budget
    b = r3.md_batch_create(int(budget))
    try:
        tickets = [r3.md_batch_submit(b, h, w.n_outer, w.k_inner, w.dt_outer) for w, h in zip(ws[:3], hs[:3])]
        r3.md_batch_run(b, 8)  # one cycle (40 ticks): the small ones finish, the large one is resident
        q, res = r3.md_batch_pending(b)
        assert (q, res) == (0, 1)
        for w, h in zip(ws[3:], hs[3:]):  # arrivals while the large member is resident
            tickets.append(r3.md_batch_submit(b, h, w.n_outer, w.k_inner, w.dt_outer))
        r3.md_batch_run(b, 8)  # admits what fits beside the large member, runs one cycle
        q, _ = r3.md_batch_pending(b)
        assert q >= 1  # a late request waited for memory
        r3.md_batch_run(b, 0)
        for w, h, t, (xa, va, f2a, f3a) in zip(ws, hs, tickets, alone):
            assert r3.md_batch_poll(b, t)
            x, v = r3.md_get_state(h)
            f2, f3 = r3.md_get_forces(h)
            ek, u2, u3, _ = r3.md_get_energy(h)
            for got, ref in ((x, xa), (v, va), (f2, f2a), (f3, f3a)):
                assert np.array_equal(got, ref)
            r2, r3f, ekr, u2r, u3r = _oracle_at(w, x, v)
            assert _force_err(f2, r2) <= 1e-5
            assert _force_err(f3, r3f) <= 1e-5
            scale = ekr + abs(u2r) + abs(u3r)
            assert abs(ek - ekr) / scale <= 1e-12
            assert abs(u2 - u2r) / scale <= 1e-6
            assert abs(u3 - u3r) / scale <= 1e-6
    finally:
        r3.md_batch_destroy(b)
        for h in hs:
            r3.md_destroy_system(h)


def test_served_fp64_follows_algorithm2(gpu_lib):
    """The FP64 served path (deferred systems, budget admission, arrivals while cycles run): every
    request's final positions and velocities follow Algorithm 2 of the oracle within 1e-10 / 1e-9."""
    r3 = gpu_lib
    ws = _systems(151)
    n_outer = 3
    hs = []
    for w in ws:
        h = r3.md_create_system(w.x, w.L, w.v, 1.0, r3.MD_FP64 | r3.MD_DEFERRED)
        r3.md_set_potentials(h, 1.0, 1.0, 2.5, NU, 2.5)
        hs.append(h)
    b = r3.md_batch_create(3 * 1024 * 1024)
    try:
        tickets = [r3.md_batch_submit(b, h, n_outer, w.k_inner, w.dt_outer) for w, h in zip(ws[:2], hs[:2])]
        r3.md_batch_run(b, 4)
        for w, h in zip(ws[2:], hs[2:]):
            tickets.append(r3.md_batch_submit(b, h, n_outer, w.k_inner, w.dt_outer))
        q, _ = r3.md_batch_pending(b)
        assert q >= 1
        r3.md_batch_run(b, 0)
        for w, h, t in zip(ws, hs, tickets):
            assert r3.md_batch_poll(b, t)
            st = respa.State(w.x.copy(), w.v.copy(), w.L)
            f2b, f3b = respa.lj_atm_forces(w.L, 1.0, 1.0, 2.5, NU, 2.5)
            respa.run(st, n_outer, w.k_inner, w.dt_outer, f2b, f3b)
            x, v = r3.md_get_state(h)
            assert _dist(x, st.x, w.L) < 1e-10
            assert np.abs(v - st.v).max() < 1e-9
    finally:
        r3.md_batch_destroy(b)
        for h in hs:
            r3.md_destroy_system(h)


def test_particle_bound_holds_requests_back(gpu_lib):
    """md_batch_set_limits: with a bound of 1800 resident particles, requests of 800 and 900 particles
    are admitted together and one of 1000 waits in the queue until they finish; a request of 2000 (more
    than the bound by itself) then runs alone.  Every request's final state equals the same request run
    alone bit for bit (FP32, rotation triplet kernel, the batch's row LJ kernel)."""
    r3 = gpu_lib
    specs = [(800, 0.8, 1.0, 4), (900, 0.8, 1.1, 4), (1000, 0.75, 1.0, 4), (2000, 0.8, 1.0, 4)]
    ws = []
    for i, (n, rho, T, k) in enumerate(specs):
        w = md_inputs.fcc_system(n, rho, T, 0.05, 731 + i)
        w.k_inner, w.dt_outer = k, 0.002 * k
        ws.append(w)
    n_outer = 3
    alone = []
    for w in ws:
        with r3.System.create(w.x, w.L, w.v, precision=0, nu=NU, atm_kernel=2, lj_kernel=0) as s:
            s.step(n_outer, w.k_inner, w.dt_outer)
            alone.append(s.state())
    hs = []
    for w in ws:
        h = r3.md_create_system(w.x, w.L, w.v, 1.0, r3.MD_FP32 | r3.MD_DEFERRED)
        r3.md_set_potentials(h, 1.0, 1.0, 2.5, NU, 2.5)
        r3.md_set_atm_kernel(h, 2)
        hs.append(h)
    b = r3.md_batch_create(0)
    try:
        with pytest.raises(r3.MDError):
            r3.md_batch_set_limits(b, -1)
        r3.md_batch_set_limits(b, 1800)
        tickets = [r3.md_batch_submit(b, h, n_outer, w.k_inner, w.dt_outer) for w, h in zip(ws[:3], hs[:3])]
        r3.md_batch_run(b, 4)  # one cycle of the first admission
        assert r3.md_batch_pending(b) == (1, 2)  # 800 + 900 resident, 1000 queued
        tickets.append(r3.md_batch_submit(b, hs[3], n_outer, ws[3].k_inner, ws[3].dt_outer))
        r3.md_batch_run(b, 0)
        for w, h, t, (xa, va) in zip(ws, hs, tickets, alone):
            assert r3.md_batch_poll(b, t)
            x, v = r3.md_get_state(h)
            assert np.array_equal(x, xa) and np.array_equal(v, va)
    finally:
        r3.md_batch_destroy(b)
        for h in hs:
            r3.md_destroy_system(h)
