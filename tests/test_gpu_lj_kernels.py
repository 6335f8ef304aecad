"""GPU parity of the LJ kernels (row kernel 0, cell-tile kernel 1, team kernel 2) against the CPU FP64
oracle.

Pair forces and energy of Sec. 2.1 (LJ 12-6, truncated at r_c2 inclusive) on grids with 3, 5 and 6
cells per side (the cell-tile kernel's blocks of 2 x 2 x 2 cells: periodic images staged twice, ragged
last blocks, whole blocks), at x0 and after outer steps (drifted cell-local coordinates), in FP32
(max relative error 1e-5, energy 1e-6) and FP64 (1e-12); and a half-empty box whose dense blocks
overflow the tile kernel's staging, so the call grows it and replays.
"""
import numpy as np
import pytest

import md_inputs
import oracle
from oracle import respa

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-12}
ETOL = {0: 1e-6, 1: 1e-12}
NU = 0.073


def force_err(got, ref):
    frms = np.sqrt((ref ** 2).sum(1).mean())
    return float((np.linalg.norm(got - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), frms)).max())


def create(r3, w, prec, lj_kernel, nu=NU):
    s = r3.System.create(w.x, w.L, w.v, precision=prec, nu=nu)
    r3.md_set_lj_kernel(s.handle, lj_kernel)
    return s


# n at density 0.8: L = 10.77 (3 cells per side), 15.54 (5), 18.42 (6)
@pytest.mark.parametrize("n", [1000, 3000, 5000])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("lj_kernel", [0, 1, 2])
def test_lj_kernels_match_oracle(gpu_lib, n, prec, lj_kernel):
    r3 = gpu_lib
    w = md_inputs.fcc_system(n, 0.8, 1.0, 0.05, md_inputs.config_seed(2, 40 + n % 97))
    f2r, u2r, w2r = oracle.lj_brute(w.x, w.L, 1.0, 1.0, 2.5)
    scale = oracle.kinetic(w.v) + abs(u2r)
    with create(r3, w, prec, lj_kernel) as s:
        f2, _ = s.forces()
        _, u2, _, _ = s.energy()
        st = s.stats()
        assert st["lj_kernel"] == lj_kernel
        assert st["cells_per_side"] == {1000: 3, 3000: 5, 5000: 6}[n]
        assert force_err(f2, f2r) <= TOL[prec]
        assert abs(u2 - u2r) / scale <= ETOL[prec]
        # after outer steps the cell-local coordinates have drifted from the cell centres
        s.step(3, 5, 0.01)
        x, _ = s.state()
        f2b, _ = s.forces()
        _, u2b, _, _ = s.energy()
    f2rb, u2rb, _ = oracle.lj_brute(x, w.L, 1.0, 1.0, 2.5)
    assert force_err(f2b, f2rb) <= TOL[prec]
    assert abs(u2b - u2rb) / scale <= ETOL[prec]


@pytest.mark.parametrize("lj_kernel", [0, 1, 2])
@pytest.mark.parametrize("prec", [0, 1])
def test_lj_kernels_follow_algorithm2(gpu_lib, prec, lj_kernel):
    """Each kernel along 4 outer steps of k = 5 against Algorithm 2 run by the oracle (positions and
    velocities within the tolerances of the single-system trajectory test)."""
    r3 = gpu_lib
    w = md_inputs.small_fcc_1k()
    st = respa.State(w.x.copy(), w.v.copy(), w.L)
    f2b, f3b = respa.lj_atm_forces(w.L, 1.0, 1.0, 2.5, NU, 2.5)
    respa.run(st, 4, 5, 0.01, f2b, f3b)
    with create(r3, w, prec, lj_kernel) as s:
        s.step(4, 5, 0.01)
        x, v = s.state()
        assert s.stats()["lj_kernel"] == lj_kernel
    d = x - st.x
    d -= w.L * np.rint(d / w.L)
    xtol, vtol = (2e-5, 2e-4) if prec == 0 else (1e-10, 1e-9)
    assert np.abs(d).max() < xtol
    assert np.abs(v - st.v).max() < vtol


def test_tile_staging_grows_on_a_half_empty_box(gpu_lib):
    """Particles on a jittered simple-cubic lattice (spacing 1) fill the slab 3 <= x < 15 of a box of
    side 24 (8 cells of edge 3 per side): 27 particles in each of the cells 1-4 along x, none in the
    others.  The block whose 4^3 region cells are cells 1-4 along x stages 64 x 27 = 1728 particles, more
    than the staging sized from the mean occupancy (52 x 27 + 64 = 1468), so the first call overflows
    it, grows the cell capacity and replays; forces and energy still equal the oracle's."""
    r3 = gpu_lib
    L = 24.0
    g = np.stack(np.meshgrid(np.arange(12), np.arange(24), np.arange(24), indexing="ij"), -1).reshape(-1, 3)
    seed = md_inputs.config_seed(2, 77)
    jit = 0.05 * md_inputs.gaussian(seed, 1, 0, 3 * len(g)).reshape(-1, 3)
    x = (g + np.array([3.5, 0.5, 0.5]) + jit) % L
    v = md_inputs.maxwell(len(x), 1.0, seed)
    f2r, u2r, _ = oracle.lj_brute(x, L, 1.0, 1.0, 2.5)
    scale = oracle.kinetic(v) + abs(u2r)  # the energy metric of every parity test
    for prec in (0, 1):
        s = r3.System.create(x, L, v, precision=prec, nu=0.0)
        try:
            r3.md_set_lj_kernel(s.handle, 1)
            f2, _ = s.forces()
            _, u2, _, _ = s.energy()
            st = s.stats()
        finally:
            s.close()
        assert st["lj_kernel"] == 1
        assert force_err(f2, f2r) <= TOL[prec]
        assert abs(u2 - u2r) / scale <= ETOL[prec]
