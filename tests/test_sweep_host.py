"""Host-side logic of the energy sweep (no GPU): RVITE (Eq. 4) and the deviation histogram of Sec. 4.2.1."""
import numpy as np
import pytest

from oracle import respa


def test_rvite_is_eq4():
    from paper_2507_11172_gb300 import sweeps
    e = np.array([1.0, 3.0, 1.0, 3.0, 2.0])
    k = np.full(5, 4.0)
    # mean 2, mean absolute deviation (1 + 1 + 1 + 1 + 0) / 5 = 0.8, divided by K = 4
    assert sweeps.rvite(e, k) == pytest.approx(0.2)
    assert sweeps.rvite(e, k) == pytest.approx(respa.rvite(e, k))


def test_deviation_histogram_pairs_equal_times():
    from paper_2507_11172_gb300 import sweeps
    s = 3
    e1 = -100.0 - np.arange(1, 31, dtype=float)  # energy after k + 1 Stormer-Verlet iterations
    # s = 3 run: after j + 1 full steps (iteration 3 (j + 1)), relative deviation 1e-3 (j + 1)
    t = 3 * np.arange(1, 11)
    es = e1[t - 1] + 1e-3 * np.arange(1, 11) * np.abs(e1[t - 1])
    counts, edges = sweeps.deviation_histogram(es, e1, s, bins=10)
    assert counts.sum() == 10 and np.all(counts == 1)
    assert edges[0] == pytest.approx(1e-3) and edges[-1] == pytest.approx(1e-2)
