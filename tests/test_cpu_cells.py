"""The linked-cell CPU baseline (cpu_cells/) against the brute-force oracle: forces, energies, triplet
counts and Algorithm 2 trajectories.  The baseline is what bench.py times as the CPU throughput figure;
these pins make sure it computes the same truncated sums (Sec. 2.1, the triplet cutoff of Fig. 2 and
Sec. 4.2.2) and the same integrator (Algorithm 2) as the oracle."""
import numpy as np
import pytest

import cpu_cells
import md_inputs
import oracle
from oracle import respa

NU = 0.073


def _err(got, ref):
    frms = np.sqrt((ref ** 2).sum(1).mean())
    return float((np.linalg.norm(got - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), frms)).max())


@pytest.mark.parametrize("rc2,rc3", [(2.5, 2.5), (2.5, 2.0), (2.0, 2.6)])
def test_forces_energies_and_count_match_brute_force(rc2, rc3):
    w = md_inputs.small_fcc_1k()
    f2, f3, o = cpu_cells.forces(w.x, w.L, 1.0, 1.0, rc2, NU, rc3)
    r2, u2, w2 = oracle.lj_brute(w.x, w.L, 1.0, 1.0, rc2)
    r3, u3, _, cnt = oracle.atm_brute(w.x, w.L, NU, rc3)
    assert o["triplets"] == cnt
    assert _err(f2, r2) <= 1e-12 and _err(f3, r3) <= 1e-12
    assert abs(o["u2"] - u2) <= 1e-12 * abs(u2) and abs(o["w2"] - w2) <= 1e-12 * abs(w2)
    assert abs(o["u3"] - u3) <= 1e-12 * abs(u3)


def test_three_cells_per_side_and_a_liquid_start():
    """The smallest grid (three cells per side: every stencil cell is a periodic neighbour on some
    axis) on a random sequential addition start."""
    n, rho = 360, 0.75
    x, L = md_inputs.rsa(n, rho, 0.85, 11)
    assert int(L // 2.5) == 3
    f2, f3, o = cpu_cells.forces(x, L)
    r2, _, _ = oracle.lj_brute(x, L, 1.0, 1.0, 2.5)
    r3, u3, _, cnt = oracle.atm_brute(x, L, NU, 2.5)
    assert o["triplets"] == cnt
    assert _err(f2, r2) <= 1e-12 and _err(f3, r3) <= 1e-12
    assert abs(o["u3"] - u3) <= 1e-12 * abs(u3)


def test_trajectory_follows_algorithm2():
    """Split calls (forces carried over) against the oracle's Algorithm 2: 3 outer steps of k = 5."""
    w = md_inputs.small_fcc_1k()
    st = respa.State(w.x.copy(), w.v.copy(), w.L)
    f2b, f3b = respa.lj_atm_forces(w.L, 1.0, 1.0, 2.5, NU, 2.5)
    respa.run(st, 3, 5, 0.01, f2b, f3b)
    c = cpu_cells.State(w.x, w.v, w.L, nu=NU)
    c.run(1, 5, 0.01)
    r = c.run(2, 5, 0.01)
    d = c.x - st.x
    d -= w.L * np.rint(d / w.L)
    assert np.abs(d).max() < 1e-12 and np.abs(c.v - st.v).max() < 1e-11
    assert abs(r["u2"] - st.u2) <= 1e-12 * abs(st.u2) and abs(r["u3"] - st.u3) <= 1e-12 * abs(st.u3)
    assert r["atm_evals"] == 2


def test_box_of_fewer_than_three_cells_is_rejected():
    x, L = md_inputs.fcc_jitter(32, 0.8, 0.05, 3)
    with pytest.raises(ValueError):
        cpu_cells.forces(x, L)


def test_empty_system():
    f2, f3, o = cpu_cells.forces(np.zeros((0, 3)), 10.0)
    assert f2.shape == (0, 3) and f3.shape == (0, 3)
    assert o["triplets"] == 0 and o["u2"] == 0.0 and o["u3"] == 0.0
    st = cpu_cells.State(np.zeros((0, 3)), np.zeros((0, 3)), 10.0)
    r = st.run(2, 3, 0.01)
    assert r["triplets"] == 0 and r["atm_evals"] == 2
