"""Failure detection without a GPU fault: every failure here is made on the host (an input that drives a
state non-finite, a request too large for the memory budget, a cancelled request), and the library must
report it through its status codes while everything else carries on:
  * a batch member that goes non-finite during a cycle fails alone (MD_ERR_NONFINITE), the other members
    finish and equal their lone runs within the FP32 tolerance of the batch tests;
  * a request that can never fit the batch's memory budget fails with MD_ERR_OOM, the others finish;
  * md_batch_cancel drops a queued request (its system untouched) and stops a resident one at the end of
    its current outer step (its state a full step of Algorithm 2, equal to a lone run of as many steps);
  * a lone system that goes non-finite returns MD_ERR_NONFINITE from md_respa_step with its state restored
    to the start of the call.
No kernel is made to fault, trap or wait: the non-finite member has one particle with a huge (finite)
velocity, so its cell-local coordinates overflow to infinity in FP32 and its LJ forces become NaN, which
the kernels flag; binning clamps every cell index, so no access leaves its array."""
import numpy as np
import pytest

import md_inputs
import oracle

pytestmark = pytest.mark.gpu

NU = 0.073
MiB = 1024 * 1024


def _w(n, rho, T, k, seed):
    w = md_inputs.fcc_system(n, rho, T, 0.05, seed)
    w.k_inner = k
    w.dt_outer = 0.002 * k
    return w


def _alone(r3, w, n_outer):
    # the LJ kernel batches use (row kernel): the same bits alone and in the batch
    with r3.System.create(w.x, w.L, w.v, precision=0, nu=NU, atm_kernel=2, lj_kernel=0) as s:
        s.step(n_outer, w.k_inner, w.dt_outer)
        return s.state()


def _dist(a, b, L):
    d = a - b
    d -= L * np.rint(d / L)
    return np.abs(d).max()


def _handle(r3, w, deferred=False):
    h = r3.md_create_system(w.x, w.L, w.v, 1.0, r3.MD_FP32 | (r3.MD_DEFERRED if deferred else 0))
    r3.md_set_potentials(h, 1.0, 1.0, 2.5, NU, 2.5)
    r3.md_set_atm_kernel(h, 2)
    return h


def test_non_finite_member_fails_alone(gpu_lib):
    r3 = gpu_lib
    ws = [_w(700, 0.8, 1.0, 4, 301), _w(900, 0.8, 1.2, 4, 302), _w(800, 0.75, 1.0, 4, 303)]
    bad = ws[1]
    bad.v = bad.v.copy()
    bad.v[0] = [1e300, 0.0, 0.0]  # finite, but its first drift leaves FP32 range
    n_outer = 3
    alone = {i: _alone(r3, ws[i], n_outer) for i in (0, 2)}
    b = r3.md_batch_create(0)
    hs = [_handle(r3, w) for w in ws]
    try:
        tickets = [r3.md_batch_submit(b, h, n_outer, w.k_inner, w.dt_outer) for w, h in zip(ws, hs)]
        r3.md_batch_run(b, 0)
        with pytest.raises(r3.MDError) as e:
            r3.md_batch_poll(b, tickets[1])
        assert e.value.status == -4
        for i in (0, 2):
            assert r3.md_batch_poll(b, tickets[i])
            x, v = r3.md_get_state(hs[i])
            xa, va = alone[i]
            assert _dist(x, xa, ws[i].L) < 1e-6
            assert np.abs(v - va).max() < 1e-5
            assert np.all(np.isfinite(x)) and np.all(np.isfinite(v))
    finally:
        r3.md_batch_destroy(b)
        for h in hs:
            r3.md_destroy_system(h)


def test_request_larger_than_the_budget_fails_with_oom(gpu_lib):
    r3 = gpu_lib
    small = [_w(600, 0.8, 1.0, 4, 311), _w(700, 0.8, 1.0, 2, 312)]
    big = _w(12000, 0.8, 1.0, 4, 313)
    n_outer = 2
    hs = [_handle(r3, small[0], True), _handle(r3, big, True), _handle(r3, small[1], True)]
    need = [r3.md_get_memory(h) for h in hs]
    budget = max(need[0], need[2]) * 3  # both small ones fit; the large one never does
    assert need[1] > budget
    alone = [_alone(r3, w, n_outer) for w in small]
    b = r3.md_batch_create(budget)
    try:
        t = [r3.md_batch_submit(b, h, n_outer, w.k_inner, w.dt_outer) for w, h in zip([small[0], big, small[1]], hs)]
        r3.md_batch_run(b, 0)
        with pytest.raises(r3.MDError) as e:
            r3.md_batch_poll(b, t[1])
        assert e.value.status == -2
        for j, (w, xa) in zip((0, 2), zip(small, alone)):
            assert r3.md_batch_poll(b, t[j])
            x, _ = r3.md_get_state(hs[j])
            assert _dist(x, xa[0], w.L) < 1e-6
        assert r3.md_batch_pending(b) == (0, 0)
    finally:
        r3.md_batch_destroy(b)
        for h in hs:
            r3.md_destroy_system(h)


def test_cancel_queued_and_resident_requests(gpu_lib):
    r3 = gpu_lib
    wa = _w(800, 0.8, 1.0, 4, 321)   # resident, cancelled after its first cycle
    wb = _w(600, 0.8, 1.0, 4, 322)   # queued behind the budget, cancelled before it runs
    ha, hb = _handle(r3, wa, True), _handle(r3, wb, True)
    b = r3.md_batch_create(r3.md_get_memory(ha) + r3.md_get_memory(hb) // 2)
    try:
        ta = r3.md_batch_submit(b, ha, 10, wa.k_inner, wa.dt_outer)
        tb = r3.md_batch_submit(b, hb, 10, wb.k_inner, wb.dt_outer)
        r3.md_batch_run(b, 4)  # one cycle (P = 4 ticks): a is one outer step in, b waits for memory
        assert r3.md_batch_pending(b) == (1, 1)
        r3.md_batch_cancel(b, tb)
        r3.md_batch_cancel(b, ta)
        r3.md_batch_run(b, 0)
        for t in (ta, tb):
            with pytest.raises(r3.MDError) as e:
                r3.md_batch_poll(b, t)
            assert e.value.status == -9
        with pytest.raises(r3.MDError) as e:
            r3.md_batch_cancel(b, ta)  # already cancelled
        assert e.value.status == -7
        steps = r3.md_batch_latency(b, ta).size
        assert 1 <= steps < 10
        xa, va = r3.md_get_state(ha)
        xr, vr = _alone(r3, wa, steps)
        assert _dist(xa, xr, wa.L) < 1e-6 and np.abs(va - vr).max() < 1e-5
        assert r3.md_get_stats(ha)["outer_steps"] == steps
        xb, vb = r3.md_get_state(hb)  # never admitted: the caller's state, folded into the box
        assert _dist(xb, wb.x, wb.L) < 1e-12 and np.array_equal(vb, wb.v)
    finally:
        r3.md_batch_destroy(b)
        r3.md_destroy_system(ha)
        r3.md_destroy_system(hb)


def test_lone_system_going_non_finite_restores_its_state(gpu_lib):
    r3 = gpu_lib
    w = _w(700, 0.8, 1.0, 4, 331)
    with r3.System.create(w.x, w.L, w.v, precision=0, nu=NU) as s:
        s.step(1, 4, 0.008)
        x0, v0 = s.state()
        v1 = v0.copy()
        v1[5] = [0.0, -1e300, 0.0]
        s.set_state(vel=v1)
        with pytest.raises(r3.MDError) as e:
            s.step(2, 4, 0.008)
        assert e.value.status == -4
        x, v = s.state()
        assert np.array_equal(x, x0) and np.array_equal(v, v1)


def test_copy_barrier_timeout_is_reported_and_the_context_survives(gpu_lib):
    """The cell-tile LJ kernel waits for its bulk shared-memory copies on an mbarrier with a bounded poll.
    A host-side knob makes the kernel announce 16 bytes more than it copies: every copy completes, the
    barrier's phase never does, the wait runs out and the call fails with MD_ERR_DEVICE_TIMEOUT; the state
    is the call's start, and the same handle goes on normally once the knob is off (forces at the final
    positions equal the oracle's)."""
    r3 = gpu_lib
    w = _w(1000, 0.8, 1.0, 4, 311)
    with r3.System.create(w.x, w.L, w.v, precision=0, nu=NU, lj_kernel=1) as s:
        s.step(1, w.k_inner, w.dt_outer)
        assert s.stats()["lj_kernel"] == 1
        x0, v0 = s.state()
        r3.md_inject_copy_shortfall(s.handle, 16)
        with pytest.raises(r3.MDError) as ei:
            s.step(1, w.k_inner, w.dt_outer)
        assert ei.value.status == -5  # MD_ERR_DEVICE_TIMEOUT
        x1, v1 = s.state()
        assert np.array_equal(x1, x0) and np.array_equal(v1, v0)
        r3.md_inject_copy_shortfall(s.handle, 0)
        s.step(2, w.k_inner, w.dt_outer)
        x, _ = s.state()
        f2, f3 = s.forces()
    sel = np.arange(0, w.n, 7)
    r2, _ = oracle.lj_particles(x, w.L, sel, 1.0, 1.0, 2.5)
    r3f, _, _ = oracle.atm_particles(x, w.L, sel, NU, 2.5)
    for got, ref in ((f2[sel], r2), (f3[sel], r3f)):
        frms = np.sqrt((ref ** 2).sum(1).mean())
        err = np.linalg.norm(got - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), frms)
        assert err.max() <= 1e-5
