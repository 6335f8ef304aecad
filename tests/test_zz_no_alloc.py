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
