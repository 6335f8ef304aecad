"""Pins for the LJ part of the oracle (Sec. 2.1) and for the r-RESPA integrator
(Algorithm 2, Sec. 4.1): closed forms, lattice sums, finite differences,
textbook special cases (s = 1 is Stormer-Verlet; nu = 0 is plain Verlet on LJ),
an exact two-force harmonic split, time reversibility and bounded energy error.
"""
import itertools
import math

import numpy as np
import pytest

import md_inputs
import oracle
from oracle import respa


def _pair(r, eps=1.3, sigma=0.9, rc=10.0):
    x = np.array([[1.0, 1.0, 1.0], [1.0 + r, 1.0, 1.0]])
    f, u, w = oracle.lj_brute(x, 40.0, eps, sigma, rc)
    return f, u, w


def test_lj_closed_forms():
    eps, sigma = 1.3, 0.9
    # phi(sigma) = 0; minimum -eps at 2^(1/6) sigma with zero force
    _, u, _ = _pair(sigma, eps, sigma)
    assert abs(u) < 1e-13  # the pair distance itself carries one rounding
    rmin = 2 ** (1 / 6) * sigma
    f, u, _ = _pair(rmin, eps, sigma)
    assert u == pytest.approx(-eps, rel=1e-14)
    assert np.abs(f).max() < 1e-13
    # pair virial r . F = 48 eps (s/r)^12 - 24 eps (s/r)^6 (from -r dphi/dr)
    for r in (0.95, 1.1, 1.7, 2.4):
        f, u, w = _pair(r, eps, sigma)
        s6 = (sigma / r) ** 6
        assert w == pytest.approx(48 * eps * s6 * s6 - 24 * eps * s6, rel=1e-13)
        assert f[1, 0] * r == pytest.approx(w, rel=1e-13)  # F_j along +x
        assert f[0, 0] == -f[1, 0]


def test_lj_fcc_and_sc_lattice_sums():
    # perfect FCC with r_c between the first two shells: 6 N bonds of length a/sqrt2
    a = 1.6
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    cells = np.array(list(itertools.product(range(3), repeat=3)), dtype=float)
    x = ((cells[:, None, :] + basis[None]) * a).reshape(-1, 3)
    n = x.shape[0]
    ann = a / math.sqrt(2)
    f, u, _ = oracle.lj_brute(x, 3 * a, 1.0, 1.0, a * 0.95)
    assert u == pytest.approx(6 * n * 4 * (ann ** -12 - ann ** -6), rel=1e-12)
    assert np.abs(f).max() < 1e-11
    # simple cubic spacing b with r_c in [b, sqrt2 b): 3 N bonds
    b = 1.15
    x = np.array(list(itertools.product(range(7), repeat=3)), dtype=float) * b
    f, u, _ = oracle.lj_brute(x, 7 * b, 1.0, 1.0, b * 1.2)
    assert u == pytest.approx(3 * x.shape[0] * 4 * (b ** -12 - b ** -6), rel=1e-12)


def test_lj_cutoff_inclusive_and_gradient():
    x = np.array([[1.0, 1.0, 1.0], [3.5, 1.0, 1.0]])
    _, u, _ = oracle.lj_brute(x, 20.0, 1.0, 1.0, 2.5)
    assert u == pytest.approx(4 * (2.5 ** -12 - 2.5 ** -6), rel=1e-14)
    x[1, 0] = np.nextafter(3.5, 4.0)
    _, u, _ = oracle.lj_brute(x, 20.0, 1.0, 1.0, 2.5)
    assert u == 0.0
    rng = np.random.default_rng(11)
    L, rc = 8.0, 2.5
    x = rng.uniform(0, L, size=(40, 3))
    f, u, _ = oracle.lj_brute(x, L, 1.0, 1.0, rc)
    d = x[None] - x[:, None]
    d -= L * np.rint(d / L)
    r = np.linalg.norm(d, axis=-1)
    h = 1e-7
    for i in range(0, 40, 3):
        if np.any(np.abs(r[i] - rc) < 1e-4):
            continue
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, c] += h
            xm[i, c] -= h
            fd = -(oracle.lj_brute(xp, L, 1.0, 1.0, rc)[1] - oracle.lj_brute(xm, L, 1.0, 1.0, rc)[1]) / (2 * h)
            assert f[i, c] == pytest.approx(fd, rel=1e-5, abs=1e-6 * np.abs(f).max())
    assert np.abs(f.sum(0)).max() < 1e-10 * np.abs(f).max()
    sel = np.arange(40)
    fp, up = oracle.lj_particles(x, L, sel, 1.0, 1.0, rc)
    assert up.sum() / 2 == pytest.approx(u, rel=1e-12)
    assert np.abs(fp - f).max() < 1e-12 * np.abs(f).max()


# ---------------------------------------------------------------- integrator

def _small_system(n=64, seed=3, rho=0.8):
    x, L = md_inputs.fcc_jitter(n, rho, 0.05, seed)
    v = md_inputs.maxwell(n, 1.0, seed)
    return x, v, L


def _velocity_verlet(x, v, L, force, dt, steps, m=1.0):
    """Textbook Stormer-Verlet (velocity form), independent of oracle.respa."""
    f = force(x)
    for _ in range(steps):
        v = v + 0.5 * dt / m * f
        x = oracle.wrap(x + dt * v, L)
        f = force(x)
        v = v + 0.5 * dt / m * f
    return x, v


def test_s1_is_stormer_verlet():
    # Sec. 4.1: step-size factor 1 "corresponds to the Stormer Verlet algorithm"
    x, v, L = _small_system()
    f2b, f3b = respa.lj_atm_forces(L, 1.0, 1.0, 2.5, 0.5, 2.5)
    st = respa.State(x.copy(), v.copy(), L)
    respa.run(st, 12, 1, 0.004, f2b, f3b)
    xv, vv = _velocity_verlet(x, v, L, lambda y: f2b(y)[0] + f3b(y)[0], 0.004, 12)
    assert np.abs(st.x - xv).max() < 1e-12
    assert np.abs(st.v - vv).max() < 1e-11


def test_nu0_is_verlet_on_lj():
    x, v, L = _small_system()
    f2b, f3b = respa.lj_atm_forces(L, 1.0, 1.0, 2.5, 0.0, 2.5)
    st = respa.State(x.copy(), v.copy(), L)
    respa.run(st, 3, 5, 0.01, f2b, f3b)
    xv, vv = _velocity_verlet(x, v, L, lambda y: f2b(y)[0], 0.002, 15)
    assert np.abs(st.x - xv).max() < 1e-12
    assert np.abs(st.v - vv).max() < 1e-11


def test_harmonic_two_force_split_matches_matrix_product():
    # 1-D oscillator split into a fast spring k0 (inner, every step) and a slow spring k1
    # (outer): one outer step is K1(h) * M0^s * K1(h), h = s dt / 2, where K1 is the kick
    # [[1, 0], [-k1 h / m, 1]] and M0 the Verlet step matrix of the fast spring.
    m, k0, k1, dt, s = 1.7, 3.0, 0.4, 0.05, 4
    K1 = np.array([[1.0, 0.0], [-k1 * s * dt / (2 * m), 1.0]])
    c = dt * dt * k0 / (2 * m)
    M0 = np.array([[1 - c, dt], [-dt * k0 / (2 * m) * (2 - c), 1 - c]])
    step = K1 @ np.linalg.matrix_power(M0, s) @ K1
    assert np.linalg.det(step) == pytest.approx(1.0, abs=1e-13)  # symplectic
    x0 = np.array([[0.8, 0.0, 0.0]])
    v0 = np.array([[-0.3, 0.0, 0.0]])

    def fast(y):
        return -k0 * y, 0.0, 0.0

    def slow(y):
        return -k1 * y, 0.0, 0.0
    st = respa.State(x0.copy(), v0.copy(), 1e9, mass=m)
    respa.run(st, 7, s, s * dt, fast, slow, periodic=False)
    want = np.linalg.matrix_power(step, 7) @ np.array([0.8, -0.3])
    assert st.x[0, 0] == pytest.approx(want[0], rel=1e-12)
    assert st.v[0, 0] == pytest.approx(want[1], rel=1e-12)


def test_time_reversibility():
    x, v, L = _small_system(n=108, seed=5)
    f2b, f3b = respa.lj_atm_forces(L, 1.0, 1.0, 2.5, 0.3, 2.5)
    st = respa.State(x.copy(), v.copy(), L)
    respa.run(st, 6, 4, 0.008, f2b, f3b)
    st.v = -st.v
    respa.run(st, 6, 4, 0.008, f2b, f3b)
    d = st.x - x
    d -= L * np.rint(d / L)
    assert np.abs(d).max() < 1e-10
    assert np.abs(st.v + v).max() < 1e-9


def _cluster_energy_error(dt_outer, n_outer, k):
    # open cluster in a large box with r_c above every distance: no pair or triplet ever
    # crosses the cutoff, so the energy error is the integrator's alone
    x, _ = md_inputs.fcc_jitter(32, 0.9, 0.05, 9)
    x = x - x.mean(0) + 50.0
    v = md_inputs.maxwell(32, 0.3, 9)
    L, rc = 200.0, 60.0
    f2b, f3b = respa.lj_atm_forces(L, 1.0, 1.0, rc, 0.073, rc)
    st = respa.State(x.copy(), v.copy(), L)
    respa.run(st, 0, k, dt_outer, f2b, f3b)
    e0 = oracle.kinetic(v) + st.u2 + st.u3
    respa.run(st, n_outer, k, dt_outer, f2b, f3b, record=True)
    e = np.array([sum(t) for t in st.energies])
    return np.abs(e - e0).max() / abs(e0)


def test_energy_error_is_second_order():
    # symplectic second-order integrator: halving the step cuts the energy error about 4x
    err1 = _cluster_energy_error(0.02, 10, 4)
    err2 = _cluster_energy_error(0.01, 20, 4)
    assert err1 < 1e-3
    assert 3.0 < err1 / err2 < 5.5


def test_periodic_energy_stays_bounded():
    # periodic, truncated potentials: the cutoff adds small energy jumps (Sec. 4.2 notes this
    # for Cutoff runs) but the total energy at full steps must stay in a narrow band with no
    # linear drift
    x, v, L = _small_system(n=256, seed=7)
    f2b, f3b = respa.lj_atm_forces(L, 1.0, 1.0, 2.5, 0.073, 2.5)
    st = respa.State(x.copy(), v.copy(), L)
    respa.run(st, 0, 4, 0.008, f2b, f3b)
    e0 = oracle.kinetic(v) + st.u2 + st.u3
    respa.run(st, 30, 4, 0.008, f2b, f3b, record=True)
    e = np.array([sum(t) for t in st.energies])
    assert np.abs(e - e0).max() / abs(e0) < 5e-3
    half = len(e) // 2
    assert np.abs(e[half:] - e0).mean() < 4 * np.abs(e[:half] - e0).mean() + 1e-12


def test_rvite_definition():
    # Eq. 4 on a series with known mean absolute deviation
    e = np.array([1.0, 3.0, 1.0, 3.0])
    k = np.array([2.0, 2.0, 2.0, 2.0])
    assert respa.rvite(e, k) == pytest.approx(0.5)
