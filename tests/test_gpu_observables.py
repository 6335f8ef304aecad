"""GPU parity of the observables: RDF pair counts (bit-exact integer counts against the oracle's
CPU histogram of the same positions) and the virial pressure."""
import numpy as np
import pytest

import md_inputs
import oracle
from oracle import observables as obs

pytestmark = pytest.mark.gpu

NU = 0.073


@pytest.mark.parametrize("prec", [0, 1])
def test_rdf_counts_match_the_oracle_exactly(gpu_lib, prec):
    w = md_inputs.small_fcc_1k()
    with gpu_lib.System.create(w.x, w.L, w.v, precision=prec, nu=NU) as s:
        for nbins, r_max in ((50, 2.5), (1000, 2.79), (7, 0.9)):
            c = s.rdf(nbins, r_max)
            x, _ = s.state()
            ref = obs.rdf_counts(x, w.L, nbins, r_max)
            assert np.array_equal(c.astype(np.int64), ref)
        # after outer steps: the positions of the last binning, their own pair list
        s.step(2, 5, 0.01)
        c = s.rdf(100, 2.5)
        x, _ = s.state()
        assert np.array_equal(c.astype(np.int64), obs.rdf_counts(x, w.L, 100, 2.5))


def test_rdf_ragged_small_box(gpu_lib):
    """37 random particles in a box of side 9 (three cells per side, wrap-around pairs)."""
    x, _ = md_inputs.rsa(37, 37 / 9.0 ** 3, 0.85, 5)
    L = 9.0
    with gpu_lib.System.create(x, L, None, precision=0) as s:
        c = s.rdf(64, 2.7)
        xs, _ = s.state()
    assert np.array_equal(c.astype(np.int64), obs.rdf_counts(xs, L, 64, 2.7))


def test_rdf_rejects_radii_beyond_the_pair_list(gpu_lib):
    w = md_inputs.small_fcc_1k()
    with gpu_lib.System.create(w.x, w.L, w.v, nu=NU) as s:
        with pytest.raises(gpu_lib.MDError):
            s.rdf(10, 3.5)
        with pytest.raises(gpu_lib.MDError):
            s.rdf(0, 2.0)


def test_100k_rdf_total_pairs(gpu_lib):
    """Full-size workload: the pair count below r_max equals an independent periodic k-d tree count
    (library routine) of the same positions, and every bin matches it."""
    spatial = pytest.importorskip("scipy.spatial")
    w = md_inputs.fcc_100k()
    nbins, r_max = 25, 2.5
    with gpu_lib.System.create(w.x, w.L, w.v, nu=NU) as s:
        c = s.rdf(nbins, r_max).astype(np.int64)
        x, _ = s.state()
    tree = spatial.cKDTree(x, boxsize=w.L)
    edges = obs.bin_edges(nbins, r_max)
    below = np.array([tree.count_neighbors(tree, np.nextafter(e, 0.0)) for e in edges[1:]])
    assert np.array_equal(np.cumsum(c), (below - len(x)) // 2)


@pytest.mark.parametrize("prec,tol", [(0, 1e-5), (1, 1e-12)])
def test_pressure_matches_the_oracle(gpu_lib, prec, tol):
    w = md_inputs.small_fcc_1k()
    _, _, w2 = oracle.lj_brute(w.x, w.L, 1.0, 1.0, 2.5)
    _, _, w3, _ = oracle.atm_brute(w.x, w.L, NU, 2.5)
    ref = obs.pressure(oracle.kinetic(w.v), w2 + w3, w.L)
    with gpu_lib.System.create(w.x, w.L, w.v, precision=prec, nu=NU) as s:
        ek, _, _, vir = s.energy()
    assert abs(obs.pressure(ek, vir, w.L) - ref) <= tol * abs(ref)
