"""Pins for the ATM part of the CPU oracle (paper Sec. 2.1, Fig. 2 caption, Sec. 4.2.2).

Nothing here re-types the oracle's formula: every expected value is a closed
form derived by hand from the potential's definition, a lattice sum counted by
hand, an invariant, or a finite difference of the oracle's own energy.
"""
import itertools
import math

import numpy as np
import pytest

import oracle

NU = 0.37


def _rand_triangle(rng, scale=1.0):
    while True:
        p = rng.normal(size=(3, 3)) * scale
        d = [np.linalg.norm(p[a] - p[b]) for a, b in ((0, 1), (0, 2), (1, 2))]
        if min(d) > 0.5 * scale:
            return p


def test_equilateral_closed_form():
    # all angles 60 deg: 1 + 3 (1/2)^3 = 11/8, so phi = 11 nu / (8 r^9); by symmetry each
    # force is radial from the centroid and sum r.F = 9 phi gives |F| = 3 sqrt(3) phi / r.
    for r in (0.9, 1.0, 1.7, 2.5):
        p = np.array([0.0, 0.0, 0.0])
        q = np.array([r, 0.0, 0.0])
        s = np.array([r / 2, r * math.sqrt(3) / 2, 0.0])
        phi, g = oracle.atm_triangle(p, q, s, NU)
        want = 11.0 * NU / (8.0 * r ** 9)
        assert phi == pytest.approx(want, rel=1e-14)
        c = (p + q + s) / 3
        for a, pt in enumerate((p, q, s)):
            f = -g[a]
            radial = (pt - c) / np.linalg.norm(pt - c)
            assert np.dot(f, radial) == pytest.approx(3 * math.sqrt(3) * want / r, rel=1e-13)
            assert np.linalg.norm(f - np.dot(f, radial) * radial) < 1e-13 * np.linalg.norm(f)


def test_collinear_closed_form():
    # points 0, a, a+b on a line: angles 0, pi, 0 so 1 + 3 cos cos cos = -2 and
    # phi = -2 nu / D^3 with D = a b (a + b); d/dx of D^-3 gives the end forces.
    for a, b in ((1.0, 1.0), (1.1, 1.7), (0.8, 2.3)):
        D = a * b * (a + b)
        pts = np.array([[0.0, 0.0, 0.0], [a, 0.0, 0.0], [a + b, 0.0, 0.0]])
        phi, g = oracle.atm_triangle(pts[0], pts[1], pts[2], NU)
        assert phi == pytest.approx(-2 * NU / D ** 3, rel=1e-13)
        f = -g
        assert f[0, 0] == pytest.approx(6 * NU * b * (2 * a + b) / D ** 4, rel=1e-12)
        assert f[2, 0] == pytest.approx(-6 * NU * a * (a + 2 * b) / D ** 4, rel=1e-12)
        assert f[1, 0] == pytest.approx(-(f[0, 0] + f[2, 0]), rel=1e-12, abs=1e-15)
        assert np.abs(f[:, 1:]).max() < 1e-14


def test_right_angle_closed_form():
    # cos(th_i) = 0 removes the angular term: phi = nu / (r_ij r_ik r_jk)^3
    for u, w in ((1.0, 1.0), (1.3, 0.7), (2.0, 1.1)):
        p, q, s = np.zeros(3), np.array([u, 0.0, 0.0]), np.array([0.0, w, 0.0])
        phi, _ = oracle.atm_triangle(p, q, s, NU)
        assert phi == pytest.approx(NU / (u * w * math.hypot(u, w)) ** 3, rel=1e-14)


def test_homogeneity_virial_and_zero_net_force():
    # phi3 is homogeneous of degree -9 in the coordinates: sum r_a . F_a = 9 phi;
    # translation invariance gives sum F = 0, rotation invariance sum r x F = 0.
    rng = np.random.default_rng(1)
    for _ in range(50):
        pts = _rand_triangle(rng)
        phi, g = oracle.atm_triangle(pts[0], pts[1], pts[2], NU)
        f = -g
        assert np.sum(pts * f) == pytest.approx(9 * phi, rel=1e-11, abs=1e-13)
        scale = np.abs(f).max()
        assert np.abs(f.sum(0)).max() < 1e-12 * scale
        assert np.abs(np.cross(pts, f).sum(0)).max() < 1e-11 * scale


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    h = 1e-6
    for _ in range(20):
        pts = _rand_triangle(rng)
        _, g = oracle.atm_triangle(pts[0], pts[1], pts[2], NU)
        for a in range(3):
            for c in range(3):
                pp, pm = pts.copy(), pts.copy()
                pp[a, c] += h
                pm[a, c] -= h
                fd = (oracle.atm_triangle(*pp, NU)[0] - oracle.atm_triangle(*pm, NU)[0]) / (2 * h)
                assert g[a, c] == pytest.approx(fd, rel=1e-6, abs=1e-8 * np.abs(g).max())


def _fcc(nc, a):
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    cells = np.array(list(itertools.product(range(nc), repeat=3)), dtype=float)
    return ((cells[:, None, :] + basis[None]) * a).reshape(-1, 3), nc * a


def test_fcc_first_shell_lattice_sum():
    # Perfect FCC, r_c between the first (a/sqrt2) and second (a) shells: every site has
    # 12 nearest neighbours, 4 of them common with each neighbour, so 12*4/2 = 24 triangles
    # per site and 8 N equilateral triangles of side a_nn in total; forces vanish by symmetry.
    a = 1.6
    x, L = _fcc(3, a)
    ann = a / math.sqrt(2)
    n = x.shape[0]
    for rc in (ann * 1.01, a * 0.99):
        f, u, w, cnt = oracle.atm_brute(x, L, NU, rc)
        assert cnt == 8 * n
        assert u == pytest.approx(8 * n * 11 * NU / (8 * ann ** 9), rel=1e-12)
        assert np.abs(f).max() < 1e-12
        assert w == pytest.approx(9 * u, rel=1e-12)


def test_simple_cubic_needs_all_three_distances():
    # Simple cubic, spacing b, r_c in [b, sqrt2 b): two nearest-neighbour bonds always meet at
    # 90 or 180 degrees, so the third side is sqrt2 b or 2b > r_c: no triplet may count even
    # though every particle has 6 neighbours within r_c.
    b = 1.2
    nc = 8
    x = np.array(list(itertools.product(range(nc), repeat=3)), dtype=float) * b
    L = nc * b
    f, u, w, cnt = oracle.atm_brute(x, L, NU, b * 1.3)
    assert cnt == 0 and u == 0.0 and np.abs(f).max() == 0.0
    # r_c in [sqrt2 b, sqrt3 b): bonds of length b and sqrt2 b.  Triangles with all sides in
    # {b, sqrt2 b}: (b, b, sqrt2 b) right isosceles -- at each site 3 pairs of perpendicular axes
    # x 4 sign choices = 12, each triangle has one right-angle vertex -> 12 N; and equilateral
    # (sqrt2 b)^3 face-diagonal triangles -- each of the 6 N face-diagonal bonds lies in 4 of
    # them -> 6 N * 4 / 3 = 8 N.  No other combination closes on the integer lattice.
    rc = b * 1.5
    f, u, w, cnt = oracle.atm_brute(x, L, NU, rc)
    n = x.shape[0]
    right = NU / (b * b * math.sqrt(2) * b) ** 3  # cos at the right angle is 0
    equi = 11 * NU / (8 * (math.sqrt(2) * b) ** 9)
    assert cnt == 12 * n + 8 * n
    assert u == pytest.approx(12 * n * right + 8 * n * equi, rel=1e-12)
    assert np.abs(f).max() < 1e-12


def test_cutoff_is_inclusive():
    # "less than or equal to the cutoff" (Fig. 2 caption, Sec. 4.2.2): a side exactly at r_c
    # counts, a side one ulp above does not.
    rc = 2.0
    L = 20.0
    base = np.array([[5.0, 5.0, 5.0], [7.0, 5.0, 5.0], [6.0, 5.0 + math.sqrt(3.0), 5.0]])
    x = base.copy()
    x[2] = [6.0, 6.0, 5.0]  # sides 2, sqrt2, sqrt2: exactly at the cutoff on the first side
    _, u_in, _, c_in = oracle.atm_brute(x, L, NU, rc)
    assert c_in == 1 and u_in != 0.0
    x2 = x.copy()
    x2[1, 0] = np.nextafter(7.0, 8.0)
    _, u_out, _, c_out = oracle.atm_brute(x2, L, NU, rc)
    assert c_out == 0 and u_out == 0.0


def test_periodic_minimum_image_matches_unwrapped():
    # a triangle straddling the box corner has the energy of its unwrapped copy in the middle
    rng = np.random.default_rng(3)
    L = 9.0
    for _ in range(10):
        tri = _rand_triangle(rng, scale=0.9)
        mid = tri + 4.5
        corner = (tri + 0.1) % L
        phi = oracle.atm_triangle(mid[0], mid[1], mid[2], NU)[0]
        f, u, _, c = oracle.atm_brute(corner, L, NU, 2.9)
        fm, um, _, cm = oracle.atm_brute(mid, L, NU, 2.9)
        assert c == cm
        if c:
            assert u == pytest.approx(phi, rel=1e-12)
            assert np.abs(f - fm).max() < 1e-11 * np.abs(fm).max()


def _random_system(n, L, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0, L, size=(n, 3))


def test_system_forces_are_minus_energy_gradient():
    L, rc = 8.0, 2.5
    x = _random_system(60, L, 4)
    dd = x[None] - x[:, None]
    dd -= L * np.rint(dd / L)
    rr = np.linalg.norm(dd, axis=-1) + np.eye(60) * 9
    x = x[rr.min(axis=1) > 0.7]
    f, u, _, _ = oracle.atm_brute(x, L, NU, rc)
    h = 1e-6
    d = x[None] - x[:, None]
    d -= L * np.rint(d / L)
    r = np.linalg.norm(d, axis=-1)
    for i in range(0, x.shape[0], 5):
        if np.any(np.abs(r[i] - rc) < 1e-4):
            continue  # a finite difference across the cutoff would measure the jump
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, c] += h
            xm[i, c] -= h
            fd = -(oracle.atm_brute(xp, L, NU, rc)[1] - oracle.atm_brute(xm, L, NU, rc)[1]) / (2 * h)
            assert f[i, c] == pytest.approx(fd, rel=2e-6, abs=1e-7 * np.abs(f).max())


def test_open_cluster_invariants():
    # box far larger than the cluster and r_c: no image, no cutoff inside the cluster
    rng = np.random.default_rng(5)
    pts = rng.uniform(0, 3.0, size=(12, 3)) + 40.0
    L, rc = 100.0, 30.0
    f, u, w, cnt = oracle.atm_brute(pts, L, NU, rc)
    assert cnt == 12 * 11 * 10 // 6
    scale = np.abs(f).max()
    assert np.abs(f.sum(0)).max() < 1e-10 * scale
    c = pts.mean(0)
    assert np.abs(np.cross(pts - c, f).sum(0)).max() < 1e-9 * scale
    # rotation: energy unchanged, forces rotate
    th = 0.7
    R = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1.0]])
    pr = (pts - c) @ R.T + c
    fr, ur, _, _ = oracle.atm_brute(pr, L, NU, rc)
    assert ur == pytest.approx(u, rel=1e-12)
    assert np.abs(fr - f @ R.T).max() < 1e-10 * scale
    # translation
    ft, ut, _, _ = oracle.atm_brute(pts + np.array([3.3, -1.1, 7.7]), L, NU, rc)
    assert ut == pytest.approx(u, rel=1e-12)
    assert w == pytest.approx(9 * u, rel=1e-10)


def test_tiny_inputs_against_itertools_enumeration():
    # independent enumeration of the triple set: every combination of 3 distinct indices,
    # tested with math.dist on explicit minimum-image copies, energy from the cosines.
    rng = np.random.default_rng(6)
    L, rc = 8.0, 2.6
    for n in (3, 4, 7, 12, 25):
        x = rng.uniform(0, L, size=(n, 3))
        _, u, _, cnt = oracle.atm_brute(x, L, NU, rc)
        uu, cc = 0.0, 0
        for i, j, k in itertools.combinations(range(n), 3):
            def img(a, b):
                return [b[t] - L * round((b[t] - a[t]) / L) for t in range(3)]
            pj = img(x[i], x[j])
            pk = img(x[i], x[k])
            pkj = img(x[j], x[k])
            if max(math.dist(x[i], pj), math.dist(x[i], pk), math.dist(x[j], pkj)) > rc:
                continue
            pts = [list(x[i]), pj, pk]
            ang = []
            for a in range(3):
                o, b1, b2 = pts[a], pts[(a + 1) % 3], pts[(a + 2) % 3]
                v1 = [b1[t] - o[t] for t in range(3)]
                v2 = [b2[t] - o[t] for t in range(3)]
                ang.append(math.acos(max(-1.0, min(1.0, sum(v1[t] * v2[t] for t in range(3)) /
                                                  (math.hypot(*v1) * math.hypot(*v2))))))
            rr = math.dist(pts[0], pts[1]) * math.dist(pts[0], pts[2]) * math.dist(pts[1], pts[2])
            uu += NU * (1 + 3 * math.cos(ang[0]) * math.cos(ang[1]) * math.cos(ang[2])) / rr ** 3
            cc += 1
        assert cnt == cc
        assert u == pytest.approx(uu, rel=1e-10, abs=1e-14)


def test_per_particle_pass_agrees_with_triple_loop():
    rng = np.random.default_rng(7)
    L, rc = 9.0, 2.5
    x = rng.uniform(0, L, size=(300, 3))
    f, u, _, cnt = oracle.atm_brute(x, L, NU, rc)
    sel = np.arange(300)
    fp, up, cp = oracle.atm_particles(x, L, sel, NU, rc)
    assert cp.sum() == 3 * cnt
    assert up.sum() / 3 == pytest.approx(u, rel=1e-12)
    assert np.abs(fp - f).max() < 1e-12 * np.abs(f).max()
