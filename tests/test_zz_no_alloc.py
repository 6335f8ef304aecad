"""Allocation-free ATM forces (md_atm_forces_noalloc) against md_get_forces.

Some callers cannot allocate device memory (a framework that owns the memory
pool, a locked-down allocator, code that must not trigger the synchronisation
of cudaMalloc/cudaFree).  The allocation-free entry point serves them with
scratch arrays that live in the library itself; here its forces, energy and
triplet count must equal those of the regular FP32 path within the FP32
tolerance (max relative per-particle force error <= 1e-5, energy <= 1e-6,
identical triplet counts), on two calls in a row with different inputs and a
third that repeats the first (the scratch keeps each call's leftovers).
"""
import numpy as np
import pytest

import md_inputs

pytestmark = pytest.mark.gpu

NU, RC = 0.073, 2.5


def _force_err(got, ref):
    frms = np.sqrt((ref ** 2).sum(1).mean())
    return float((np.linalg.norm(got - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), frms)).max())


def _regular(r3, w):
    with r3.System.create(w.x, w.L, w.v, precision=r3.MD_FP32, nu=NU, rc_triplet=RC) as s:
        _, f3 = s.forces()
        _, _, u3, _ = s.energy()
        cnt = s.stats()["triplets_last"]
    return f3, u3, cnt


def test_noalloc_matches_regular_entry_point(gpu_lib):
    import torch
    r3 = gpu_lib
    systems = [md_inputs.small_fcc_1k(), md_inputs.fcc_system(4000, 0.85, 1.2, 0.05, md_inputs.config_seed(9))]
    refs = [_regular(r3, w) for w in systems]
    for idx in (0, 1, 0):  # two calls in a row, then the first input again
        w = systems[idx]
        f_ref, u_ref, c_ref = refs[idx]
        d_pos = torch.from_numpy(np.ascontiguousarray(w.x)).cuda()
        d_f3 = torch.full_like(d_pos, float("nan"))
        u3, cnt = r3.md_atm_forces_noalloc(d_pos.data_ptr(), w.n, w.L, NU, RC, d_f3.data_ptr())
        f3 = d_f3.cpu().numpy()
        assert cnt == c_ref
        assert _force_err(f3, f_ref) <= 1e-5
        assert abs(u3 - u_ref) <= 1e-6 * abs(u_ref)


def test_noalloc_rejects_sizes_above_its_limit(gpu_lib):
    r3 = gpu_lib
    with pytest.raises(r3.MDError) as e:
        r3.md_atm_forces_noalloc(1, 16385, 40.0, NU, RC, 1)  # rejected before any device access
    assert e.value.status == -8


def _oracle_atm(w):
    import oracle
    allp = np.arange(w.n)
    f, u, c = oracle.atm_particles(w.x, w.L, allp, NU, RC)
    return f, u.sum() / 3, int(c.sum()) // 3


def test_noalloc_matches_the_oracle_and_clamps_coarse_cells(gpu_lib):
    """The allocation-free entry point against the oracle's per-particle pass directly (every particle):
    on the 1,000-particle FCC system, and in a sparse box whose cell grid the entry point clamps to
    32^3 cells (L = 90 > 32 r_c: two dense FCC blocks of 1,000 particles far apart, open surfaces), where
    it must also agree with md_get_forces.  Forces within 1e-5, energy within 1e-6, counts exact."""
    import torch
    r3 = gpu_lib
    a = md_inputs.small_fcc_1k()
    b = md_inputs.fcc_system(1000, 0.8, 1.0, 0.05, md_inputs.config_seed(9, 3))
    sparse = md_inputs.Workload(name="two_blocks_L90", x=np.concatenate([a.x + 5.0, b.x + 50.0]),
                                v=np.zeros((2000, 3)), L=90.0)
    for w in (a, sparse):
        f_ref, u_ref, c_ref = _oracle_atm(w)
        d_pos = torch.from_numpy(np.ascontiguousarray(w.x)).cuda()
        d_f3 = torch.full_like(d_pos, float("nan"))
        u3, cnt = r3.md_atm_forces_noalloc(d_pos.data_ptr(), w.n, w.L, NU, RC, d_f3.data_ptr())
        f3 = d_f3.cpu().numpy()
        assert cnt == c_ref
        assert _force_err(f3, f_ref) <= 1e-5
        assert abs(u3 - u_ref) <= 1e-6 * abs(u_ref)
    f_reg, u_reg, c_reg = _regular(r3, sparse)
    assert c_reg == c_ref and _force_err(f_reg, f_ref) <= 1e-5
