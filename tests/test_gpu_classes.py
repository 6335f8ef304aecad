"""GPU parity of the distance classes of the three-body force (near triplets within an intermediate
cutoff r_a integrated every s_near inner steps, far triplets every outer step) against the oracle's
three-level r-RESPA (oracle.respa.run3) and its class forces.  Tolerances as for Algorithm 2."""
import numpy as np
import pytest

import md_inputs
import oracle
from oracle import respa

pytestmark = pytest.mark.gpu

NU = 0.073
TOL = {0: 1e-5, 1: 1e-12}


def force_err(got, ref):
    frms = np.sqrt((ref ** 2).sum(1).mean())
    return float((np.linalg.norm(got - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), max(frms, 1e-300))).max())


@pytest.fixture(scope="module")
def cfg1():
    return md_inputs.small_fcc_1k()


def make(r3, w, prec, r_a, s_near, skin=None, kernel=-1):
    s = r3.System.create(w.x, w.L, w.v, precision=prec, nu=NU, skin=skin, atm_kernel=kernel)
    s.set_distance_classes(r_a, s_near)
    return s


def oracle_run3(w, n_outer, k, s_near, dt_outer, r_a):
    f2b, _ = respa.lj_atm_forces(w.L, 1.0, 1.0, 2.5, NU, 2.5)
    near, far = respa.class_forces(w.L, NU, r_a, 2.5)
    st = respa.State3(w.x.copy(), w.v.copy(), w.L)
    respa.run3(st, n_outer, k, s_near, dt_outer, f2b, near, far)
    return st


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("r_a", [1.3, 1.8, 2.5])
def test_class_forces_and_counts_at_x0(gpu_lib, cfg1, prec, r_a):
    f3r, _, _, cnt = oracle.atm_brute(cfg1.x, cfg1.L, NU, 2.5)
    f3nr, _, _, cntn = oracle.atm_brute(cfg1.x, cfg1.L, NU, r_a)
    with make(gpu_lib, cfg1, prec, r_a, 2) as s:
        _, f3 = s.forces()
        f3n = s.near_forces()
        st = s.stats()
    assert st["triplets_last"] == cnt and st["near_triplets_last"] == cntn
    assert force_err(f3, f3r) <= TOL[prec]
    assert force_err(f3n, f3nr) <= TOL[prec]


@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_every_triplet_kernel_with_classes(gpu_lib, cfg1, kernel):
    """The whole ATM force comes from any of the three triplet kernels; the near class from its own."""
    st = oracle_run3(cfg1, 2, 4, 2, 0.008, 1.8)
    with make(gpu_lib, cfg1, 1, 1.8, 2, kernel=kernel) as s:
        s.step(2, 4, 0.008)
        x, v = s.state()
        assert s.stats()["atm_kernel"] == kernel
    d = x - st.x
    d -= cfg1.L * np.rint(d / cfg1.L)
    assert np.abs(d).max() < 1e-10 and np.abs(v - st.v).max() < 1e-9


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("k,s_near", [(6, 2), (6, 3), (4, 1)])
def test_trajectory_matches_three_level_oracle(gpu_lib, cfg1, prec, k, s_near):
    """4 outer steps in two calls (forces cached across them); near lists rebuilt between binnings."""
    dt_outer, r_a = 0.002 * k, 1.8
    st = oracle_run3(cfg1, 4, k, s_near, dt_outer, r_a)
    with make(gpu_lib, cfg1, prec, r_a, s_near) as s:
        s.step(1, k, dt_outer)
        s.step(3, k, dt_outer)
        x, v = s.state()
        f2, f3 = s.forces()
        f3n = s.near_forces()
        stats = s.stats()
    d = x - st.x
    d -= cfg1.L * np.rint(d / cfg1.L)
    xtol, vtol = (2e-5, 2e-4) if prec == 0 else (1e-10, 1e-9)
    assert np.abs(d).max() < xtol
    assert np.abs(v - st.v).max() < vtol
    ftol = 1e-4 if prec == 0 else 1e-9  # forces at slightly different positions
    assert force_err(f3n, st.f3n) < ftol
    assert force_err(f3, st.f3n + st.f3f) < ftol
    assert force_err(f2, st.f2) < ftol
    assert stats["outer_steps"] == 4


def test_one_near_block_per_outer_step_equals_algorithm2(gpu_lib, cfg1):
    """s_near = k: the near and far kicks fall together, i.e. Algorithm 2 with the whole force."""
    with make(gpu_lib, cfg1, 1, 1.8, 5) as a:
        a.step(3, 5, 0.01)
        xa, va = a.state()
    with gpu_lib.System.create(cfg1.x, cfg1.L, cfg1.v, precision=1, nu=NU, atm_kernel=2) as b:
        b.step(3, 5, 0.01)
        xb, vb = b.state()
    d = xa - xb
    d -= cfg1.L * np.rint(d / cfg1.L)
    assert np.abs(d).max() < 1e-11 and np.abs(va - vb).max() < 1e-10


def test_empty_far_class_is_algorithm2_with_the_near_factor(gpu_lib, cfg1):
    """r_a = r_c3: every triplet is near, so 3 outer steps of k = 6 with s_near = 2 are 9 outer
    steps of Algorithm 2 with k = 2."""
    with make(gpu_lib, cfg1, 1, 2.5, 2) as a:
        a.step(3, 6, 0.012)
        xa, va = a.state()
    with gpu_lib.System.create(cfg1.x, cfg1.L, cfg1.v, precision=1, nu=NU, atm_kernel=2) as b:
        b.step(9, 2, 0.004)
        xb, vb = b.state()
    d = xa - xb
    d -= cfg1.L * np.rint(d / cfg1.L)
    assert np.abs(d).max() < 1e-11 and np.abs(va - vb).max() < 1e-10


@pytest.mark.parametrize("n,L", [(37, 9.0), (300, 9.0), (777, 10.0), (1283, 11.7)])
def test_ragged_sizes(gpu_lib, n, L):
    x, L = md_inputs.fcc_jitter(n, n / L ** 3, 0.08, n)
    f3r, _, _, cnt = oracle.atm_brute(x, L, NU, 2.5)
    f3nr, _, _, cntn = oracle.atm_brute(x, L, NU, 1.9)
    with gpu_lib.System.create(x, L, None, precision=1, nu=NU) as s:
        s.set_distance_classes(1.9, 1)
        _, f3 = s.forces()
        f3n = s.near_forces()
        st = s.stats()
    assert st["triplets_last"] == cnt and st["near_triplets_last"] == cntn
    assert force_err(f3, f3r) <= 1e-12 and force_err(f3n, f3nr) <= 1e-12


def test_skin_violation_replays_exactly(gpu_lib, cfg1):
    """A tiny skin forces replays with a binning on every inner step; the trajectory still matches."""
    st = oracle_run3(cfg1, 2, 4, 2, 0.008, 1.8)
    with make(gpu_lib, cfg1, 1, 1.8, 2, skin=0.002) as s:
        s.step(2, 4, 0.008)
        x, v = s.state()
        assert s.stats()["replays"] >= 1
    d = x - st.x
    d -= cfg1.L * np.rint(d / cfg1.L)
    assert np.abs(d).max() < 1e-10 and np.abs(v - st.v).max() < 1e-9


def test_momentum_is_conserved(gpu_lib, cfg1):
    with make(gpu_lib, cfg1, 0, 1.5, 2) as s:
        _, v0 = s.state()
        s.step(5, 10, 0.02)
        _, v = s.state()
    assert np.abs(v.sum(0) - v0.sum(0)).max() < 1e-4


def test_errors_and_switching_off(gpu_lib, cfg1):
    r3 = gpu_lib
    with make(r3, cfg1, 1, 1.8, 2) as s:
        with pytest.raises(r3.MDError) as e:
            s.step(1, 5, 0.01)  # 5 is not a multiple of s_near = 2
        assert e.value.status == -1
        with pytest.raises(r3.MDError):
            s.set_distance_classes(2.6, 2)  # above r_c
        with pytest.raises(r3.MDError):
            s.set_distance_classes(1.8, 0)
        b = r3.md_batch_create(0)
        try:
            with pytest.raises(r3.MDError):
                r3.md_batch_submit(b, s.handle, 1, 4, 0.008)
        finally:
            r3.md_batch_destroy(b)
        s.step(1, 4, 0.008)
        s.set_distance_classes(0.0, 0)  # off again: plain Algorithm 2 from the current state
        with pytest.raises(r3.MDError):
            s.near_forces()
        x0, v0 = s.state()
        s.step(2, 4, 0.008)
        x, v = s.state()
    ref = respa.State(x0.copy(), v0.copy(), cfg1.L)
    f2b, f3b = respa.lj_atm_forces(cfg1.L, 1.0, 1.0, 2.5, NU, 2.5)
    respa.run(ref, 2, 4, 0.008, f2b, f3b)
    d = x - ref.x
    d -= cfg1.L * np.rint(d / cfg1.L)
    assert np.abs(d).max() < 1e-10


@pytest.fixture(scope="module")
def cfg2():
    return md_inputs.fcc_100k()


@pytest.mark.parametrize("prec,tol", [(0, 1e-5), (1, 1e-12)])
def test_100k_class_forces_after_steps(gpu_lib, cfg2, prec, tol):
    """100,000 particles (the benchmark's workload), r_a = 1.5, k = 10, s_near = 2: after 2 outer steps
    the cached near and whole ATM forces of a seeded 2,000-particle subset equal the oracle's at the
    GPU's own positions; total momentum is conserved."""
    u = md_inputs.uniform(md_inputs.config_seed(2), 9, 0, 4000)
    sub = np.unique((u * cfg2.n).astype(np.int64))[:2000]
    with gpu_lib.System.create(cfg2.x, cfg2.L, cfg2.v, precision=prec, nu=NU) as s:
        s.set_distance_classes(1.5, 2)
        s.step(2, 10, 0.02)
        x, v = s.state()
        _, f3 = s.forces()
        f3n = s.near_forces()
    rn, _, _ = oracle.atm_particles(x, cfg2.L, sub, NU, 1.5)
    ra, _, _ = oracle.atm_particles(x, cfg2.L, sub, NU, 2.5)
    assert force_err(f3n[sub], rn) <= tol
    assert force_err(f3[sub], ra) <= tol
    assert np.abs(v.sum(0) - cfg2.v.sum(0)).max() < (1e-3 if prec == 0 else 1e-9)


def test_too_many_near_candidates_is_a_capacity_error(gpu_lib):
    """At density 1.7 a particle has about 55 neighbours above it within r_a + skin = 2.6: more than
    the 64 candidate slots for many particles.  The call reports MD_ERR_CAPACITY (no fallback for the
    near class) and leaves the state as it was."""
    x, L = md_inputs.fcc_jitter(1500, 1.7, 0.02, 91)
    with gpu_lib.System.create(x, L, None, precision=0, nu=NU, skin=0.1) as s:
        s.set_distance_classes(2.5, 2)
        x0, v0 = s.state()
        with pytest.raises(gpu_lib.MDError) as e:
            s.step(1, 4, 0.002)
        assert e.value.status == -8
        x1, v1 = s.state()
    assert np.array_equal(x0, x1) and np.array_equal(v0, v1)
