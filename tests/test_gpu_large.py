"""Full-size parity: 100,000 particles (FCC, density 0.8, jitter 0.05, LJ r_c 2.5, ATM nu 0.073,
r_c 2.5), in the launch configuration the benchmark times.  The oracle's per-particle pass gives
exact forces of a seeded 2,000-particle subset and, over all particles, the total energies and
the interacting-triplet count."""
import numpy as np
import pytest

import md_inputs
import oracle

pytestmark = pytest.mark.gpu

NU = 0.073


def force_err(got, ref, frms):
    return float((np.linalg.norm(got - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), frms)).max())


@pytest.fixture(scope="module")
def cfg2():
    return md_inputs.fcc_100k()


@pytest.fixture(scope="module")
def subset(cfg2):
    u = md_inputs.uniform(md_inputs.config_seed(2), 9, 0, 4000)
    return np.unique((u * cfg2.n).astype(np.int64))[:2000]


@pytest.fixture(scope="module")
def full_ref(cfg2):
    allp = np.arange(cfg2.n)
    f3, u3, c3 = oracle.atm_particles(cfg2.x, cfg2.L, allp, NU, 2.5)
    f2, u2 = oracle.lj_particles(cfg2.x, cfg2.L, allp, 1.0, 1.0, 2.5)
    return dict(f2=f2, f3=f3, u2=u2.sum() / 2, u3=u3.sum() / 3, cnt=int(c3.sum()) // 3,
                frms2=np.sqrt((f2 ** 2).sum(1).mean()), frms3=np.sqrt((f3 ** 2).sum(1).mean()),
                ek=oracle.kinetic(cfg2.v))


@pytest.mark.parametrize("prec,tol", [(0, 1e-5), (1, 1e-12)])
def test_100k_forces_energy_count_at_x0(gpu_lib, cfg2, subset, full_ref, prec, tol):
    with gpu_lib.System.create(cfg2.x, cfg2.L, cfg2.v, precision=prec, nu=NU) as s:
        f2, f3 = s.forces()
        ek, u2, u3, _ = s.energy()
        cnt = s.stats()["triplets_last"]
    R = full_ref
    assert cnt == R["cnt"]
    assert force_err(f2[subset], R["f2"][subset], R["frms2"]) <= tol
    assert force_err(f3[subset], R["f3"][subset], R["frms3"]) <= tol
    # every particle, not only the subset
    assert force_err(f3, R["f3"], R["frms3"]) <= tol
    assert force_err(f2, R["f2"], R["frms2"]) <= tol
    scale = R["ek"] + abs(R["u2"]) + abs(R["u3"])
    assert abs(u2 - R["u2"]) / scale <= (1e-6 if prec == 0 else 1e-12)
    assert abs(u3 - R["u3"]) / scale <= (1e-6 if prec == 0 else 1e-12)


@pytest.mark.parametrize("prec,tol", [(0, 1e-5), (1, 1e-12)])
def test_100k_forces_after_steps(gpu_lib, cfg2, subset, prec, tol):
    """After 3 outer steps (k = 10, dt_outer = 0.02) the cached forces equal the oracle's at the
    GPU's own final positions (subset)."""
    with gpu_lib.System.create(cfg2.x, cfg2.L, cfg2.v, precision=prec, nu=NU) as s:
        s.step(3, 10, 0.02)
        x, _ = s.state()
        f2, f3 = s.forces()
    r3f, _, _ = oracle.atm_particles(x, cfg2.L, subset, NU, 2.5)
    r2f, _ = oracle.lj_particles(x, cfg2.L, subset, 1.0, 1.0, 2.5)
    assert force_err(f3[subset], r3f, np.sqrt((r3f ** 2).sum(1).mean())) <= tol
    assert force_err(f2[subset], r2f, np.sqrt((r2f ** 2).sum(1).mean())) <= tol


@pytest.fixture(scope="module")
def cfg3():
    return md_inputs.rsa_2m(2.5)


@pytest.mark.parametrize("rc3", [2.0, 2.5])
def test_2m_rsa_subset_forces_at_x0_and_after_steps(gpu_lib, cfg3, rc3):
    """2,000,000 particles, random-sequential-addition start at density 0.75, T* = 1.2, FP32 path, triplet
    cutoff 2.0 and 2.5: the forces of a seeded 300-particle subset equal the oracle's per-particle pass
    at x0 and, after 2 outer steps (k = 10, dt_outer = 0.02), at the GPU's own positions; total momentum
    is conserved."""
    u = md_inputs.uniform(md_inputs.config_seed(3), 9, 0, 600)
    sub = np.unique((u * cfg3.n).astype(np.int64))[:300]
    with gpu_lib.System.create(cfg3.x, cfg3.L, cfg3.v, precision=0, nu=NU, rc_triplet=rc3) as s:
        f2, f3 = s.forces()
        r3f, _, _ = oracle.atm_particles(cfg3.x, cfg3.L, sub, NU, rc3)
        r2f, _ = oracle.lj_particles(cfg3.x, cfg3.L, sub, 1.0, 1.0, 2.5)
        assert force_err(f3[sub], r3f, np.sqrt((r3f ** 2).sum(1).mean())) <= 1e-5
        assert force_err(f2[sub], r2f, np.sqrt((r2f ** 2).sum(1).mean())) <= 1e-5
        s.step(2, 10, 0.02)
        x, v = s.state()
        f2, f3 = s.forces()
    r3f, _, _ = oracle.atm_particles(x, cfg3.L, sub, NU, rc3)
    r2f, _ = oracle.lj_particles(x, cfg3.L, sub, 1.0, 1.0, 2.5)
    assert force_err(f3[sub], r3f, np.sqrt((r3f ** 2).sum(1).mean())) <= 1e-5
    assert force_err(f2[sub], r2f, np.sqrt((r2f ** 2).sum(1).mean())) <= 1e-5
    assert np.abs(v.sum(0) - cfg3.v.sum(0)).max() < 1e-2
