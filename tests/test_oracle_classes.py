"""Pins of the distance-class r-RESPA oracle (three levels: LJ, near triplets, far triplets; and
several classes, each with its own step-size factor)."""
import itertools

import numpy as np
import pytest

import md_inputs
import oracle
from oracle import respa


def _system(n=64, seed=3, rho=0.8):
    x, L = md_inputs.fcc_jitter(n, rho, 0.05, seed)
    v = md_inputs.maxwell(n, 1.0, seed + 1)
    return x, v, L


def test_classes_partition_the_triplets():
    """Near = all three distances <= r_a, far = the rest within r_c: counted independently by a
    plain loop over all triples."""
    x, _, L = _system(40)
    r_a, r_c = 1.8, 2.5
    d = x[:, None, :] - x[None, :, :]
    d -= L * np.rint(d / L)
    r = np.sqrt((d ** 2).sum(-1))
    near = far = 0
    for i, j, k in itertools.combinations(range(len(x)), 3):
        m = max(r[i, j], r[i, k], r[j, k])
        near += m <= r_a
        far += r_a < m <= r_c
    assert oracle.atm_brute(x, L, 0.3, r_a)[3] == near
    assert oracle.atm_brute(x, L, 0.3, r_c)[3] - near == far


def _runs(k_inner, s_near, r_a, n_outer=3, dt_outer=0.012, nu=0.4):
    x, v, L = _system()
    f2b, _ = respa.lj_atm_forces(L, 1.0, 1.0, 2.5, nu, 2.5)
    near, far = respa.class_forces(L, nu, r_a, 2.5)
    st = respa.State3(x.copy(), v.copy(), L)
    respa.run3(st, n_outer, k_inner, s_near, dt_outer, f2b, near, far)
    return x, v, L, st


def test_one_near_block_per_outer_step_is_algorithm2():
    """s_near = k_inner: near and far kicks fall on the same iterations, so the method is
    Algorithm 2 with the whole ATM force."""
    x, v, L, st = _runs(4, 4, 1.9)
    f2b, f3b = respa.lj_atm_forces(L, 1.0, 1.0, 2.5, 0.4, 2.5)
    ref = respa.State(x.copy(), v.copy(), L)
    respa.run(ref, 3, 4, 0.012, f2b, f3b)
    assert np.abs(st.x - ref.x).max() < 1e-12 and np.abs(st.v - ref.v).max() < 1e-11


def test_no_far_triplets_is_algorithm2_with_the_near_factor():
    """r_a = r_c: the far class is empty; the near triplets (all of them) are integrated with
    s_near, i.e. Algorithm 2 with s = s_near."""
    x, v, L, st = _runs(6, 2, 2.5)
    f2b, f3b = respa.lj_atm_forces(L, 1.0, 1.0, 2.5, 0.4, 2.5)
    ref = respa.State(x.copy(), v.copy(), L)
    respa.run(ref, 9, 2, 0.004, f2b, f3b)
    assert np.abs(st.x - ref.x).max() < 1e-12 and np.abs(st.v - ref.v).max() < 1e-11


def test_no_near_triplets_is_algorithm2_with_the_outer_factor():
    """r_a below the nearest-neighbour distance: no near triplets, so the near kicks vanish and
    the method is Algorithm 2 with s = k_inner."""
    x, v, L, st = _runs(6, 2, 0.5)
    f2b, f3b = respa.lj_atm_forces(L, 1.0, 1.0, 2.5, 0.4, 2.5)
    ref = respa.State(x.copy(), v.copy(), L)
    respa.run(ref, 3, 6, 0.012, f2b, f3b)
    assert np.abs(st.x - ref.x).max() < 1e-12 and np.abs(st.v - ref.v).max() < 1e-11


def test_harmonic_three_force_split_matches_nested_matrix_product():
    """1-D oscillator with three springs k0 (every step), k1 (every s_near steps), k2 (every
    k_inner steps): one outer step is K2(H) [K1(h) M0^s_near K1(h)]^(k/s_near) K2(H), written from
    the nested loops of r-RESPA (Sec. 2.3.1), not from the single loop."""
    m, k0, k1, k2, dt, s, k = 1.3, 3.0, 0.7, 0.2, 0.03, 2, 6
    def kick(kk, h):
        return np.array([[1.0, 0.0], [-kk * h / m, 1.0]])
    drift = np.array([[1.0, dt], [0.0, 1.0]])
    M0 = kick(k0, dt / 2) @ drift @ kick(k0, dt / 2)  # velocity Verlet, matrices act on (x, v)
    mid = kick(k1, s * dt / 2) @ np.linalg.matrix_power(M0, s) @ kick(k1, s * dt / 2)
    outer = kick(k2, k * dt / 2) @ np.linalg.matrix_power(mid, k // s) @ kick(k2, k * dt / 2)
    y0 = np.array([0.8, -0.3])
    st = respa.State3(np.array([[y0[0], 0.0, 0.0]]), np.array([[y0[1], 0.0, 0.0]]), 1e9, mass=m)
    lin = lambda kk: (lambda x: (-kk * x, 0.5 * kk * float((x ** 2).sum()), 0.0))
    respa.run3(st, 5, k, s, k * dt, lin(k0), lin(k1), lin(k2), periodic=False)
    y = np.linalg.matrix_power(outer, 5) @ y0
    assert abs(st.x[0, 0] - y[0]) < 1e-13 and abs(st.v[0, 0] - y[1]) < 1e-13


def test_time_reversibility():
    x, v, L = _system()
    f2b, _ = respa.lj_atm_forces(L, 1.0, 1.0, 2.5, 0.4, 2.5)
    near, far = respa.class_forces(L, 0.4, 1.9, 2.5)
    st = respa.State3(x.copy(), v.copy(), L)
    respa.run3(st, 4, 4, 2, 0.008, f2b, near, far)
    st.v = -st.v
    respa.run3(st, 4, 4, 2, 0.008, f2b, near, far)
    d = st.x - x
    d -= L * np.rint(d / L)
    assert np.abs(d).max() < 1e-10 and np.abs(st.v + v).max() < 1e-9


# ---------------------------------------------------------------- several classes

def test_two_classes_are_run3_bit_for_bit():
    x, v, L = _system()
    f2b, _ = respa.lj_atm_forces(L, 1.0, 1.0, 2.5, 0.4, 2.5)
    near, far = respa.class_forces(L, 0.4, 1.9, 2.5)
    a = respa.State3(x.copy(), v.copy(), L)
    respa.run3(a, 3, 6, 2, 0.012, f2b, near, far)
    b = respa.StateN(x.copy(), v.copy(), L)
    respa.run_classes(b, 3, 6, [2, 6], 0.012, f2b, respa.band_forces(L, 0.4, [1.9, 2.5]))
    assert np.array_equal(a.x, b.x) and np.array_equal(a.v, b.v)


def test_three_bands_partition_the_triplets():
    x, _, L = _system(40)
    cut = [1.4, 1.9, 2.5]
    fb = respa.band_forces(L, 0.3, cut)
    fall, uall, _, _ = oracle.atm_brute(x, L, 0.3, 2.5)
    fs = [f(x) for f in fb]
    assert np.abs(sum(r[0] for r in fs) - fall).max() < 1e-12 * max(1.0, np.abs(fall).max())
    assert abs(sum(r[1] for r in fs) - uall) < 1e-12 * max(1.0, abs(uall))
    # the bands' triplet counts against a plain loop over all triples
    d = x[:, None, :] - x[None, :, :]
    d -= L * np.rint(d / L)
    r = np.sqrt((d ** 2).sum(-1))
    counts = [0, 0, 0]
    for i, j, k in itertools.combinations(range(len(x)), 3):
        mx = max(r[i, j], r[i, k], r[j, k])
        for c, rc in enumerate(cut):
            if mx <= rc:
                counts[c] += 1
                break
    got = [oracle.atm_brute(x, L, 0.3, rc)[3] for rc in cut]
    assert [got[0], got[1] - got[0], got[2] - got[1]] == counts


def test_all_factors_equal_k_is_algorithm2():
    x, v, L = _system()
    f2b, f3b = respa.lj_atm_forces(L, 1.0, 1.0, 2.5, 0.4, 2.5)
    a = respa.StateN(x.copy(), v.copy(), L)
    respa.run_classes(a, 3, 4, [4, 4, 4], 0.008, f2b, respa.band_forces(L, 0.4, [1.4, 1.9, 2.5]))
    b = respa.State(x.copy(), v.copy(), L)
    respa.run(b, 3, 4, 0.008, f2b, f3b)
    assert np.abs(a.x - b.x).max() < 1e-12 and np.abs(a.v - b.v).max() < 1e-11


def test_four_spring_nested_matrix_product():
    """1-D oscillator: spring k0 every step, k1 every s1, k2 every s2, k3 every k steps; one outer step is
    K3 [K2 [K1 M0^s1 K1]^(s2/s1) K2]^(k/s2) K3 (nested loops of Sec. 2.3.1)."""
    m, dt, s1, s2, k = 1.1, 0.02, 2, 4, 8
    ks = [2.5, 0.9, 0.4, 0.1]

    def kick(kk, h):
        return np.array([[1.0, 0.0], [-kk * h / m, 1.0]])
    drift = np.array([[1.0, dt], [0.0, 1.0]])
    M0 = kick(ks[0], dt / 2) @ drift @ kick(ks[0], dt / 2)
    M1 = kick(ks[1], s1 * dt / 2) @ np.linalg.matrix_power(M0, s1) @ kick(ks[1], s1 * dt / 2)
    M2 = kick(ks[2], s2 * dt / 2) @ np.linalg.matrix_power(M1, s2 // s1) @ kick(ks[2], s2 * dt / 2)
    M3 = kick(ks[3], k * dt / 2) @ np.linalg.matrix_power(M2, k // s2) @ kick(ks[3], k * dt / 2)
    y0 = np.array([0.7, 0.2])
    st = respa.StateN(np.array([[y0[0], 0.0, 0.0]]), np.array([[y0[1], 0.0, 0.0]]), 1e9, mass=m)
    lin = lambda kk: (lambda x: (-kk * x, 0.5 * kk * float((x ** 2).sum()), 0.0))
    respa.run_classes(st, 3, k, [s1, s2, k], k * dt, lin(ks[0]), [lin(ks[1]), lin(ks[2]), lin(ks[3])],
                      periodic=False)
    y = np.linalg.matrix_power(M3, 3) @ y0
    assert abs(st.x[0, 0] - y[0]) < 1e-13 and abs(st.v[0, 0] - y[1]) < 1e-13


def test_three_classes_time_reversible():
    x, v, L = _system()
    f2b, _ = respa.lj_atm_forces(L, 1.0, 1.0, 2.5, 0.4, 2.5)
    fb = respa.band_forces(L, 0.4, [1.4, 1.9, 2.5])
    st = respa.StateN(x.copy(), v.copy(), L)
    respa.run_classes(st, 2, 4, [1, 2, 4], 0.008, f2b, fb)
    st.v = -st.v
    respa.run_classes(st, 2, 4, [1, 2, 4], 0.008, f2b, fb)
    d = st.x - x
    d -= L * np.rint(d / L)
    assert np.abs(d).max() < 1e-10 and np.abs(st.v + v).max() < 1e-9


def test_bad_class_factors_are_rejected():
    x, v, L = _system()
    f2b, _ = respa.lj_atm_forces(L, 1.0, 1.0, 2.5, 0.4, 2.5)
    fb = respa.band_forces(L, 0.4, [1.9, 2.5])
    with pytest.raises(ValueError):
        respa.run_classes(respa.StateN(x.copy(), v.copy(), L), 1, 6, [4, 6], 0.012, f2b, fb)
    with pytest.raises(ValueError):
        respa.band_forces(L, 0.4, [2.5, 1.9])
