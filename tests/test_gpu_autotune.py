"""The autotuner (launch shapes and triplet kernel, tuned on a system's first evaluation): its choices
are cached per key, so a second system with the same key skips the trials and takes the same choices;
every launch shape it can choose gives forces equal bit for bit to every other and to the oracle within
the FP32 tolerance."""
import itertools

import numpy as np
import pytest

import md_inputs
import oracle

pytestmark = pytest.mark.gpu

NU = 0.073
SKIN = 0.277  # a skin no other test uses: the cache key is new in this process


def force_err(got, ref):
    frms = np.sqrt((ref ** 2).sum(1).mean())
    return float((np.linalg.norm(got - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), frms)).max())


def test_second_system_with_the_same_key_takes_the_cached_choices(gpu_lib):
    r3 = gpu_lib
    w1 = md_inputs.fcc_system(6000, 0.8, 1.0, 0.05, 401)
    w2 = md_inputs.fcc_system(6100, 0.8, 1.0, 0.05, 402)  # same N bucket and density bucket
    with r3.System.create(w1.x, w1.L, w1.v, precision=0, nu=NU, skin=SKIN) as s1:
        f2a, f3a = s1.forces()
        st1 = s1.stats()
    with r3.System.create(w2.x, w2.L, w2.v, precision=0, nu=NU, skin=SKIN) as s2:
        s2.forces()
        st2 = s2.stats()
    assert st1["tuned_from_cache"] == 0 and st2["tuned_from_cache"] == 1
    for k in ("atm_kernel", "atm_bases_per_warp", "lj_block", "list_warps", "lj_kernel", "lj_team"):
        assert st1[k] == st2[k], k
    assert st1["lj_block"] in (32, 64, 128) and st1["list_warps"] in (2, 4, 8)
    assert st1["lj_kernel"] in (0, 1, 2) and st1["lj_team"] in (4, 8, 16)
    allp = np.arange(w1.n)
    r2, _ = oracle.lj_particles(w1.x, w1.L, allp, 1.0, 1.0, 2.5)
    r3f, _, _ = oracle.atm_particles(w1.x, w1.L, allp, NU, 2.5)
    assert force_err(f2a, r2) <= 1e-5 and force_err(f3a, r3f) <= 1e-5


def test_every_launch_shape_gives_the_same_forces(gpu_lib):
    r3 = gpu_lib
    w = md_inputs.fcc_system(3000, 0.8, 1.0, 0.05, 411)
    allp = np.arange(w.n)
    r2, _ = oracle.lj_particles(w.x, w.L, allp, 1.0, 1.0, 2.5)
    r3f, _, _ = oracle.atm_particles(w.x, w.L, allp, NU, 2.5)
    ref = None
    for lj, lw, rp in itertools.product((32, 64, 128), (2, 4, 8), (4, 16)):
        with r3.System.create(w.x, w.L, w.v, precision=0, nu=NU, atm_kernel=2) as s:
            r3.md_set_shapes(s.handle, lj, lw, rp)
            s.step(2, 4, 0.008)
            x, v = s.state()
            f2, f3 = s.forces()
            st = s.stats()
        assert (st["lj_block"], st["list_warps"], st["atm_bases_per_warp"]) == (lj, lw, rp)
        if ref is None:
            ref = (x, v, f2, f3)
            with r3.System.create(w.x, w.L, w.v, precision=0, nu=NU, atm_kernel=2) as s0:
                f20, f30 = s0.forces()
            assert force_err(f20, r2) <= 1e-5 and force_err(f30, r3f) <= 1e-5
        else:
            for a, b in zip((x, v, f2, f3), ref):
                assert np.array_equal(a, b)
    with pytest.raises(r3.MDError):
        with r3.System.create(w.x, w.L, w.v, precision=0, nu=NU) as s:
            r3.md_set_shapes(s.handle, 48, 0, 0)
