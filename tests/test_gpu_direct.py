"""All-triplet (DirectSum) ATM forces with open boundaries and no cutoff against the oracle's
brute-force triple loop (the oracle's minimum image and cutoff are neutralised by a box and a
cutoff far larger than the cluster)."""
import numpy as np
import pytest

import md_inputs
import oracle

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-12}
FAR = 1e9  # oracle box and cutoff: no image, every triplet


def force_err(got, ref):
    frms = np.sqrt((ref ** 2).sum(1).mean())
    return float((np.linalg.norm(got - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), frms)).max())


def cluster(n, rho, seed):
    """A compact open cluster: FCC + jitter, without periodic images."""
    x, _ = md_inputs.fcc_jitter(n, rho, 0.05, seed)
    return x


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n", [3, 37, 300, 701])
def test_direct_sum_matches_the_oracle(gpu_lib, n, prec):
    x = cluster(n, 0.8, 40 + n)
    nu = 0.3095  # the aluminium scenario's nu (Table 1)
    f, u = gpu_lib.md_atm_direct(x, nu, prec)
    fr, ur, _, cnt = oracle.atm_brute(x, FAR, nu, FAR)
    assert cnt == n * (n - 1) * (n - 2) // 6
    assert force_err(f, fr) <= TOL[prec]
    assert abs(u - ur) <= (1e-6 if prec == 0 else 1e-12) * abs(ur)
    # Newton 3 over the whole cluster
    assert np.abs(f.sum(0)).max() <= (1e-4 if prec == 0 else 1e-10) * np.abs(f).sum(0).max()


def test_direct_sum_of_an_equilateral_triangle(gpu_lib):
    """Closed form (Sec. 2.1): phi = 11 nu / (8 r^9), radial forces of magnitude 3 sqrt(3) phi / r."""
    r = 1.3
    x = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0], [r / 2, r * np.sqrt(3) / 2, 0.0]])
    for prec in (0, 1):
        f, u = gpu_lib.md_atm_direct(x, 1.0, prec)
        phi = 11.0 / (8.0 * r ** 9)
        assert abs(u - phi) <= 1e-6 * phi
        c = x.mean(0)
        for a in range(3):
            radial = (x[a] - c) / np.linalg.norm(x[a] - c)
            fa = 3 * np.sqrt(3) * phi / r
            assert np.linalg.norm(f[a] - fa * radial) <= 1e-5 * fa


def test_direct_sum_rejects_bad_input(gpu_lib):
    with pytest.raises(gpu_lib.MDError):
        gpu_lib.md_atm_direct(np.zeros((2, 3)), 1.0)
    with pytest.raises(gpu_lib.MDError):
        gpu_lib.md_atm_direct(np.zeros((20000, 3)), 1.0)
