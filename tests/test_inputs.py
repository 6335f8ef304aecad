"""Synthetic input recipes: FCC + vacancies + jitter, Maxwell velocities, RSA."""
import math

import numpy as np

import md_inputs


def test_fcc_vacancies_and_density():
    x, L = md_inputs.fcc_jitter(1000, 0.8, 0.0, 1)
    assert x.shape == (1000, 3)
    assert L == (1000 / 0.8) ** (1 / 3)
    # 7^3 cells x 4 sites = 1372 sites, 372 vacancies; unjittered sites sit on the lattice
    a = L / 7
    frac = (x / (a / 2)) - np.rint(x / (a / 2))
    assert np.abs(frac).max() < 1e-9
    assert len({tuple(np.round(p, 6)) for p in x}) == 1000
    x2, _ = md_inputs.fcc_jitter(1000, 0.8, 0.0, 1)
    assert np.array_equal(x, x2)  # seeded
    xj, _ = md_inputs.fcc_jitter(1000, 0.8, 0.05, 1)
    assert np.all((xj >= 0) & (xj < L))


def test_maxwell_exact_temperature_zero_momentum():
    v = md_inputs.maxwell(500, 1.2, 3)
    assert np.abs(v.sum(0)).max() < 1e-10
    assert float(np.sum(v * v)) / (3 * 500 - 3) == __import__("pytest").approx(1.2, rel=1e-12)


def test_rsa_min_distance():
    x, L = md_inputs.rsa(3000, 0.75, 0.9, 5)
    assert x.shape == (3000, 3) and math.isclose(L, (3000 / 0.75) ** (1 / 3))
    d = x[None] - x[:, None]
    d -= L * np.rint(d / L)
    r = np.linalg.norm(d, axis=-1) + np.eye(3000) * 10
    assert r.min() >= 0.9
    x2, _ = md_inputs.rsa(3000, 0.75, 0.9, 5)
    assert np.array_equal(x, x2)


def test_ensemble_specs_ranges():
    specs = md_inputs.ensemble_specs(256)
    n = np.array([s["n"] for s in specs])
    assert n.min() >= 500 and n.max() <= 20000
    assert {s["k"] for s in specs} <= {4, 8, 16}
    assert all(0.6 <= s["rho"] <= 0.9 and 0.8 <= s["T"] <= 1.5 for s in specs)
