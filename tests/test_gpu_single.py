"""GPU parity: the CUDA path through the C ABI against the CPU FP64 oracle.

Tolerances (force error e_i = |F_i - F_i^ref| / max(|F_i^ref|, F_rms^ref),
checked separately for the LJ and the ATM field):
  FP32 path (FP32 forces, compensated accumulation): max_i e_i <= 1e-5
  FP64 path: max_i e_i <= 1e-12
  energies: |E - E_ref| / (E_kin + |U2| + |U3|) <= 1e-6
Interacting-triplet counts are integers and must match exactly.
"""
import numpy as np
import pytest

import md_inputs
import oracle
from oracle import respa

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-12}
NU = 0.073


def force_err(got, ref):
    frms = np.sqrt((ref ** 2).sum(1).mean())
    floor = max(frms, 1e-300)
    return float((np.linalg.norm(got - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), floor)).max())


def make(r3, w, prec, nu=NU, rc2=2.5, rc3=2.5, skin=None, kernel=-1):
    return r3.System.create(w.x, w.L, w.v, precision=prec, nu=nu, rc_pair=rc2, rc_triplet=rc3, skin=skin,
                            atm_kernel=kernel)


@pytest.fixture(scope="module")
def cfg1():
    return md_inputs.small_fcc_1k()


@pytest.fixture(scope="module")
def cfg1_ref(cfg1):
    f2, u2, w2 = oracle.lj_brute(cfg1.x, cfg1.L, 1.0, 1.0, 2.5)
    f3, u3, w3, cnt = oracle.atm_brute(cfg1.x, cfg1.L, NU, 2.5)
    return dict(f2=f2, u2=u2, w2=w2, f3=f3, u3=u3, w3=w3, cnt=cnt, ek=oracle.kinetic(cfg1.v))


@pytest.mark.parametrize("prec", [0, 1])
def test_forces_and_energy_at_x0(gpu_lib, cfg1, cfg1_ref, prec):
    r3 = gpu_lib
    with make(r3, cfg1, prec) as s:
        f2, f3 = s.forces()
        ek, u2, u3, w = s.energy()
        st = s.stats()
    ref = cfg1_ref
    assert force_err(f2, ref["f2"]) <= TOL[prec]
    assert force_err(f3, ref["f3"]) <= TOL[prec]
    assert st["triplets_last"] == ref["cnt"]
    scale = ref["ek"] + abs(ref["u2"]) + abs(ref["u3"])
    etol = 1e-6 if prec == 0 else 1e-12
    assert abs(u2 - ref["u2"]) / scale <= etol
    assert abs(u3 - ref["u3"]) / scale <= etol
    assert abs(ek - ref["ek"]) / scale <= 1e-12
    assert abs(w - (ref["w2"] + ref["w3"])) / (abs(ref["w2"]) + abs(ref["w3"])) <= 10 * etol


@pytest.mark.parametrize("prec", [0, 1])
def test_trajectory_matches_algorithm2(gpu_lib, cfg1, prec):
    """10 outer steps of k = 5 (dt_outer = 0.01): positions, velocities, forces, energy."""
    r3 = gpu_lib
    st = respa.State(cfg1.x.copy(), cfg1.v.copy(), cfg1.L)
    f2b, f3b = respa.lj_atm_forces(cfg1.L, 1.0, 1.0, 2.5, NU, 2.5)
    respa.run(st, 10, 5, 0.01, f2b, f3b)
    with make(r3, cfg1, prec) as s:
        s.step(4, 5, 0.01)  # split calls: forces are cached across calls
        s.step(6, 5, 0.01)
        x, v = s.state()
        f2, f3 = s.forces()
        ek, u2, u3, _ = s.energy()
        stats = s.stats()
    d = x - st.x
    d -= cfg1.L * np.rint(d / cfg1.L)
    xtol, vtol = (2e-5, 2e-4) if prec == 0 else (1e-10, 1e-9)
    assert np.abs(d).max() < xtol
    assert np.abs(v - st.v).max() < vtol
    ftol = 1e-4 if prec == 0 else 1e-9  # forces at slightly different positions
    assert force_err(f2, st.f2) < ftol and force_err(f3, st.f3) < ftol
    e_ref = oracle.kinetic(st.v) + st.u2 + st.u3
    scale = oracle.kinetic(st.v) + abs(st.u2) + abs(st.u3)
    assert abs(ek + u2 + u3 - e_ref) / scale <= (1e-6 if prec == 0 else 1e-10)
    assert stats["outer_steps"] == 10 and stats["atm_evals"] == 11


@pytest.mark.parametrize("k", [1, 3])
def test_step_size_factor_variants(gpu_lib, cfg1, k):
    """k = 1 is Stormer-Verlet on F2 + F3 (Sec. 4.1); odd k exercises the buffer parity."""
    r3 = gpu_lib
    st = respa.State(cfg1.x.copy(), cfg1.v.copy(), cfg1.L)
    f2b, f3b = respa.lj_atm_forces(cfg1.L, 1.0, 1.0, 2.5, NU, 2.5)
    respa.run(st, 3, k, 0.002 * k, f2b, f3b)
    with make(r3, cfg1, 1) as s:
        s.step(1, k, 0.002 * k)
        s.step(2, k, 0.002 * k)
        x, v = s.state()
    d = x - st.x
    d -= cfg1.L * np.rint(d / cfg1.L)
    assert np.abs(d).max() < 1e-10 and np.abs(v - st.v).max() < 1e-9


@pytest.mark.parametrize("kernel", [-1, 2])
@pytest.mark.parametrize("n,L", [(37, 9.0), (300, 9.0), (777, 10.0), (1283, 11.7)])
def test_ragged_sizes_and_densities(gpu_lib, n, L, kernel):
    rng = np.random.default_rng(n)
    x, _ = md_inputs.rsa(n, n / L ** 3, 0.85, 100 + n)
    L = (n / (n / L ** 3)) ** (1 / 3)
    v = np.zeros_like(x)
    f2r, u2r, _ = oracle.lj_brute(x, L, 1.0, 1.0, 2.5)
    f3r, u3r, _, cnt = oracle.atm_brute(x, L, 0.5, 2.5)
    for prec in (0, 1):
        with gpu_lib.System.create(x, L, v, precision=prec, nu=0.5, atm_kernel=kernel) as s:
            f2, f3 = s.forces()
            assert s.stats()["triplets_last"] == cnt
        if cnt:
            assert force_err(f3, f3r) <= TOL[prec]
        assert force_err(f2, f2r) <= TOL[prec]
    del rng


@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_distances_exactly_at_the_cutoff(gpu_lib, kernel):
    """Simple cubic lattice, spacing 1.25, r_c = 2.5: pairs and collinear triplets sit exactly
    on the cutoff; both sides must include them (r <= r_c) and agree on the count."""
    b, m = 1.25, 8
    g = np.arange(m) * b
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).copy()
    L = m * b
    x[5] += [0.01, 0.0, 0.0]  # break the lattice symmetry a little
    f3r, u3r, _, cnt = oracle.atm_brute(x, L, NU, 2.5)
    f2r, u2r, _ = oracle.lj_brute(x, L, 1.0, 1.0, 2.5)
    for prec in (0, 1):
        with gpu_lib.System.create(x, L, None, precision=prec, nu=NU, skin=0.1, atm_kernel=kernel) as s:
            f2, f3 = s.forces()
            _, u2, u3, _ = s.energy()
            assert s.stats()["triplets_last"] == cnt
            assert s.stats()["guard_rechecks"] > 0
        # nearly every net force cancels to ~0 on this lattice, so errors are measured against
        # the scale of one triplet's force at the lattice spacing, 9 nu / b^10 (virial identity)
        scale = 9 * NU / b ** 10
        err3 = np.linalg.norm(f3 - f3r, axis=1) / np.maximum(np.linalg.norm(f3r, axis=1), scale)
        assert err3.max() <= TOL[prec]
        s6 = b ** -6
        pair_scale = abs(24 * (2 * s6 * s6 - s6) / b)  # one LJ pair at the lattice spacing
        err2 = np.linalg.norm(f2 - f2r, axis=1) / np.maximum(np.linalg.norm(f2r, axis=1), pair_scale)
        assert err2.max() <= TOL[prec]
        assert abs(u3 - u3r) <= 1e-6 * abs(u3r) + 1e-12


def test_nu_zero_gives_zero_triplet_force(gpu_lib, cfg1):
    with make(gpu_lib, cfg1, 0, nu=0.0) as s:
        _, f3 = s.forces()
        _, _, u3, _ = s.energy()
    assert np.all(f3 == 0.0) and u3 == 0.0


def test_skin_violation_replays_exactly(gpu_lib, cfg1):
    """A tiny skin makes particles leave it within an outer step; the call is replayed with a
    list rebuild on every inner step, so the trajectory still matches Algorithm 2."""
    st = respa.State(cfg1.x.copy(), cfg1.v.copy(), cfg1.L)
    f2b, f3b = respa.lj_atm_forces(cfg1.L, 1.0, 1.0, 2.5, NU, 2.5)
    respa.run(st, 3, 5, 0.01, f2b, f3b)
    with make(gpu_lib, cfg1, 1, skin=0.002) as s:
        s.step(3, 5, 0.01)
        x, v = s.state()
        assert s.stats()["replays"] >= 1
    d = x - st.x
    d -= cfg1.L * np.rint(d / cfg1.L)
    assert np.abs(d).max() < 1e-10


@pytest.mark.parametrize("skin", [0.01, 0.03, 0.06])
def test_replays_with_thin_skins_follow_algorithm2(gpu_lib, cfg1, skin):
    """Skins at which particles leave mid-call (not necessarily on the first drift): the replay restores
    the call's start and bins adaptively; consecutive calls that start in safe mode too.  Positions after
    6 outer steps in 3 calls equal Algorithm 2's."""
    st = respa.State(cfg1.x.copy(), cfg1.v.copy(), cfg1.L)
    f2b, f3b = respa.lj_atm_forces(cfg1.L, 1.0, 1.0, 2.5, NU, 2.5)
    respa.run(st, 6, 5, 0.01, f2b, f3b)
    with make(gpu_lib, cfg1, 1, skin=skin) as s:
        for _ in range(3):
            s.step(2, 5, 0.01)
        x, v = s.state()
    d = x - st.x
    d -= cfg1.L * np.rint(d / cfg1.L)
    assert np.abs(d).max() < 1e-10 and np.abs(v - st.v).max() < 1e-9


@pytest.mark.parametrize("kernel", [-1, 2])
def test_dense_cluster_grows_cell_capacity(gpu_lib, kernel):
    """All particles in one corner of a large box: cells overflow their first capacity, the
    library grows it and replays; results must still match the oracle."""
    xc, Lc = md_inputs.fcc_jitter(400, 1.0, 0.05, 77)
    L = 30.0
    x = xc + 1.0
    f3r, _, _, cnt = oracle.atm_brute(x, L, NU, 2.5)
    f2r, _, _ = oracle.lj_brute(x, L, 1.0, 1.0, 2.5)
    with gpu_lib.System.create(x, L, None, precision=0, nu=NU, atm_kernel=kernel) as s:
        f2, f3 = s.forces()
        assert s.stats()["triplets_last"] == cnt
    assert force_err(f2, f2r) <= 1e-5 and force_err(f3, f3r) <= 1e-5


@pytest.mark.parametrize("prec", [0, 1])
def test_half_lists_of_33_to_64_nodes(gpu_lib, prec):
    """At density 1.15 a particle has about 75 neighbours within r_c = 2.5, so most half lists
    (the neighbours above it) hold 33 to 64 nodes: the rotation kernel splits them into two
    halves (rotations within each half and across the halves).  Forces, energy and the exact
    triplet count must match the oracle, and the rotation kernel must stay selected."""
    x, L = md_inputs.fcc_jitter(1000, 1.15, 0.05, 93)
    f3r, u3r, _, cnt = oracle.atm_brute(x, L, NU, 2.5)
    with gpu_lib.System.create(x, L, None, precision=prec, nu=NU, skin=0.1, atm_kernel=2) as s:
        _, f3 = s.forces()
        _, _, u3, _ = s.energy()
        st = s.stats()
    assert st["atm_kernel"] == 2
    assert st["triplets_last"] == cnt
    assert force_err(f3, f3r) <= TOL[prec]
    assert abs(u3 - u3r) <= (1e-6 if prec == 0 else 1e-12) * abs(u3r)


def test_long_half_lists_fall_back_to_the_cell_kernel(gpu_lib):
    """At density 1.7 some of 1500 particles have more than 64 neighbours within r_c = 2.5 on
    their side, more than the rotation kernel's half list holds: the call is replayed with the
    cell kernel and the results still match the oracle.  (At most 122 neighbours in all, so
    even a particle of the cell kernel's first cell, which sees every neighbour as following
    it, stays within that kernel's 128-entry list.)"""
    x, L = md_inputs.fcc_jitter(1500, 1.7, 0.02, 91)
    f3r, u3r, _, cnt = oracle.atm_brute(x, L, NU, 2.5)
    with gpu_lib.System.create(x, L, None, precision=0, nu=NU, skin=0.1, atm_kernel=2) as s:
        _, f3 = s.forces()
        assert s.stats()["triplets_last"] == cnt
        assert s.stats()["atm_kernel"] == 0
        s.step(1, 2, 0.001)
        assert s.stats()["atm_kernel"] == 0
    assert force_err(f3, f3r) <= 1e-5


@pytest.mark.parametrize("prec", [0, 1])
def test_long_pair_rows(gpu_lib, prec):
    """With r_c2 = 3.5 at density 1.15 a pair-list row (list radius 3.8) holds about 260 entries, four
    times the benchmark's rows, and the triplet half lists (r_c3 = 2.5) are built from the first part of
    each row's distance range only.  LJ and ATM forces, the energies and the exact triplet count must
    match the oracle."""
    x, L = md_inputs.fcc_jitter(5324, 1.15, 0.05, 95)  # 4 cells per side of edge 4.17
    d = x[:200, None, :] - x[None, :, :]
    d -= L * np.rint(d / L)
    assert ((d ** 2).sum(2) <= 3.5 ** 2).sum(1).min() > 190
    f2r, u2r, _ = oracle.lj_brute(x, L, 1.0, 1.0, 3.5)
    f3r, u3r, _, cnt = oracle.atm_brute(x, L, NU, 2.5)
    with gpu_lib.System.create(x, L, None, precision=prec, nu=NU, rc_pair=3.5, rc_triplet=2.5, skin=0.3) as s:
        f2, f3 = s.forces()
        _, u2, u3, _ = s.energy()
        assert s.stats()["triplets_last"] == cnt
    assert force_err(f2, f2r) <= TOL[prec] and force_err(f3, f3r) <= TOL[prec]
    etol = 1e-6 if prec == 0 else 1e-12
    assert abs(u2 - u2r) <= etol * abs(u2r) and abs(u3 - u3r) <= etol * abs(u3r)


def test_errors_are_reported(gpu_lib, cfg1):
    r3 = gpu_lib
    bad = cfg1.x.copy()
    bad[3, 1] = np.nan
    with pytest.raises(r3.MDError) as e:
        r3.System.create(bad, cfg1.L)
    assert e.value.status == -4
    with pytest.raises(r3.MDError) as e:
        r3.System.create(cfg1.x, 7.0)
    assert e.value.status == -3
    with make(r3, cfg1, 0) as s:
        with pytest.raises(r3.MDError) as e:
            s.step(1, 0, 0.01)
        assert e.value.status == -1
        with pytest.raises(r3.MDError):
            r3.md_set_potentials(s.handle, 1.0, 1.0, 3.6, NU, 2.5)  # 3 * (3.6 + skin) > L


def test_checkpoint_resume(gpu_lib, cfg1):
    """Run A: 5 outer steps.  Run B: 3 steps, save state, new handle, 2 steps."""
    r3 = gpu_lib
    with make(r3, cfg1, 1) as a:
        a.step(5, 4, 0.008)
        xa, va = a.state()
    with make(r3, cfg1, 1) as b:
        b.step(3, 4, 0.008)
        xb, vb = b.state()
    with r3.System.create(xb, cfg1.L, vb, precision=1, nu=NU) as c:
        c.step(2, 4, 0.008)
        xc, vc = c.state()
    d = xc - xa
    d -= cfg1.L * np.rint(d / cfg1.L)
    assert np.abs(d).max() < 1e-11 and np.abs(vc - va).max() < 1e-10


@pytest.mark.parametrize("prec,ptol", [(0, 1e-4), (1, 1e-9)])
def test_momentum_and_energy_conservation(gpu_lib, cfg1, prec, ptol):
    with make(gpu_lib, cfg1, prec) as s:
        ek0, u20, u30, _ = s.energy()
        p0 = s.state()[1].sum(0)
        s.step(20, 5, 0.01)
        ek, u2, u3, _ = s.energy()
        p = s.state()[1].sum(0)
    e0, e1 = ek0 + u20 + u30, ek + u2 + u3
    assert np.abs(p - p0).max() < ptol  # Newton 3: pair and triplet forces sum to zero
    assert abs(e1 - e0) / (ek0 + abs(u20) + abs(u30)) < 5e-3  # truncated potentials: bounded jumps only


@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("prec", [0, 1])
def test_both_triplet_kernels_match_oracle(gpu_lib, cfg1, cfg1_ref, variant, prec):
    """Cell kernel with Newton-3 scatter (0), per-particle kernel (1) and rotation kernel (2):
    same forces, energy and interacting-triplet count as the oracle, at x0 and after a few
    outer steps."""
    r3 = gpu_lib
    with make(r3, cfg1, prec) as s:
        r3.md_set_atm_kernel(s.handle, variant)
        f2, f3 = s.forces()
        _, u2, u3, _ = s.energy()
        st = s.stats()
        assert st["atm_kernel"] == variant
        assert st["triplets_last"] == cfg1_ref["cnt"]
        assert force_err(f3, cfg1_ref["f3"]) <= TOL[prec]
        scale = cfg1_ref["ek"] + abs(cfg1_ref["u2"]) + abs(cfg1_ref["u3"])
        assert abs(u3 - cfg1_ref["u3"]) / scale <= (1e-6 if prec == 0 else 1e-12)
        s.step(2, 5, 0.01)
        x, _ = s.state()
        _, f3b = s.forces()
    sel = np.arange(0, cfg1.n, 3)
    r3f, _, _ = oracle.atm_particles(x, cfg1.L, sel, NU, 2.5)
    frms = np.sqrt((r3f ** 2).sum(1).mean())
    err = np.linalg.norm(f3b[sel] - r3f, axis=1) / np.maximum(np.linalg.norm(r3f, axis=1), frms)
    assert err.max() <= TOL[prec]


@pytest.mark.parametrize("prec", [0, 1])
def test_autotuned_rotation_shape_matches_oracle(gpu_lib, cfg1, cfg1_ref, prec):
    """Whatever kernel and work-item shape the autotuner keeps, forces and the triplet count equal the
    oracle's, before and after a call."""
    with make(gpu_lib, cfg1, prec) as s:
        _, f3 = s.forces()
        st = s.stats()
        assert st["triplets_last"] == cfg1_ref["cnt"]
        assert force_err(f3, cfg1_ref["f3"]) <= TOL[prec]
        s.step(1, 5, 0.01)
        assert s.stats()["atm_kernel"] in (0, 1, 2)
