"""Pins of the observables oracle (RDF pair counts, virial pressure) against things the paper and
the mathematics fix, not against its own formulas."""
import numpy as np
import pytest

import md_inputs
import oracle
from oracle import observables as obs


def test_rdf_counts_equal_an_independent_periodic_tree_count():
    """Cumulative pair counts at every bin edge from scipy's periodic k-d tree (a library routine,
    an independent enumeration) equal the oracle's histogram, bin by bin."""
    spatial = pytest.importorskip("scipy.spatial")
    x, L = md_inputs.fcc_jitter(600, 0.8, 0.05, 5)
    nbins, r_max = 50, 2.5
    c = obs.rdf_counts(x, L, nbins, r_max)
    tree = spatial.cKDTree(np.mod(x, L), boxsize=L)
    edges = obs.bin_edges(nbins, r_max)
    # pairs with r < edge (strict): count_neighbors counts r <= edge, so use the next float below
    below = np.array([tree.count_neighbors(tree, np.nextafter(e, 0.0)) for e in edges[1:]])
    cum = (below - len(x)) // 2  # ordered pairs incl. self -> unordered pairs
    assert np.array_equal(np.cumsum(c), cum)


def test_rdf_of_a_perfect_fcc_lattice_is_its_shell_counts():
    """Unjittered FCC (a = 1.6, n = 4 * 5^3): the pair counts are exactly the shell coordination
    numbers 12, 6, 24, 12 (times N / 2) in the bins holding a/sqrt(2), a, a sqrt(3/2), a sqrt(2)."""
    nc, a = 5, 1.6
    base = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    g = np.stack(np.meshgrid(np.arange(nc), np.arange(nc), np.arange(nc), indexing="ij"), -1).reshape(-1, 3)
    x = ((g[:, None, :] + base[None, :, :]) * a).reshape(-1, 3)
    L, n = nc * a, len(x)
    nbins, r_max = 250, 2.5
    c = obs.rdf_counts(x, L, nbins, r_max)
    edges = obs.bin_edges(nbins, r_max)
    for r_shell, z in ((a / np.sqrt(2), 12), (a, 6), (a * np.sqrt(1.5), 24), (a * np.sqrt(2), 12)):
        b = np.searchsorted(edges, r_shell, side="right") - 1
        assert c[b - 1:b + 2].sum() == z * n // 2  # rounding of the shell radius may pick a neighbour bin
    assert c.sum() == (12 + 6 + 24 + 12) * n // 2


def test_rdf_of_uniform_points_is_flat():
    """Uniform random points (an ideal gas): g(r) = 1 within the Poisson scatter of each bin."""
    u = md_inputs.uniform(3, 1, 0, 3 * 4000).reshape(-1, 3)
    L = 16.0
    x = u * L
    c = obs.rdf_counts(x, L, 10, 4.0)
    g = obs.rdf_normalise(c, len(x), L, 4.0)
    sigma = 1.0 / np.sqrt(np.maximum(c, 1))
    assert np.all(np.abs(g[2:] - 1.0) < 5 * sigma[2:] + 0.02)


def test_virial_pressure_is_minus_the_volume_derivative():
    """Homothetic scaling x -> s x, L -> s L at fixed scaled coordinates: the configurational part
    of the pressure, W / (3 V), equals -dU/dV (central differences of the oracle's energies), for
    the LJ and the ATM terms separately (both potentials are sums of powers of distances)."""
    x, L = md_inputs.fcc_jitter(300, 0.8, 0.08, 9)
    _, u2, w2 = oracle.lj_brute(x, L, 1.0, 1.0, 2.5)
    _, u3, w3, _ = oracle.atm_brute(x, L, 0.3, 2.5)
    h = 1e-6
    def energies(s):
        _, a, _ = oracle.lj_brute(x * s, L * s, 1.0, 1.0, 2.5)
        _, b, _, _ = oracle.atm_brute(x * s, L * s, 0.3, 2.5)
        return a, b
    up, um = energies(1 + h), energies(1 - h)
    V = L ** 3
    dV = V * ((1 + h) ** 3 - (1 - h) ** 3)
    for k, w in ((0, w2), (1, w3)):
        dUdV = (up[k] - um[k]) / dV
        assert abs(w / (3 * V) + dUdV) <= 1e-6 * abs(w / (3 * V)) + 1e-12


def test_ideal_gas_pressure():
    """No interactions: P = N T / V with T = 2 E_kin / (3 N)."""
    n, L, T = 500, 10.0, 1.3
    assert obs.pressure(1.5 * n * T, 0.0, L) == pytest.approx(n * T / L ** 3, rel=1e-15)
