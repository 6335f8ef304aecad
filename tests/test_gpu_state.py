"""State transfer through the C ABI (md_set_state / md_get_state / md_get_forces), which permutes between
the caller's order and the cell-sorted layout on the device: round trips, partial updates, folding into
the box, rejection of non-finite input without any change, and forces after a partial update against
the oracle."""
import numpy as np
import pytest

import md_inputs
import oracle

pytestmark = pytest.mark.gpu

NU = 0.073


@pytest.fixture(scope="module")
def cfg1():
    return md_inputs.small_fcc_1k()


def test_round_trip_after_steps_keeps_caller_order(gpu_lib, cfg1):
    with gpu_lib.System.create(cfg1.x, cfg1.L, cfg1.v, precision=1, nu=NU) as s:
        s.step(2, 5, 0.01)  # the layout is now cell-sorted
        x, v = s.state()
        s.set_state(x, v)
        x2, v2 = s.state()
    assert np.array_equal(x, x2) and np.array_equal(v, v2)
    assert np.all((x >= 0) & (x < cfg1.L))


def test_partial_updates(gpu_lib, cfg1):
    rng = np.random.default_rng(5)
    with gpu_lib.System.create(cfg1.x, cfg1.L, cfg1.v, precision=1, nu=NU) as s:
        s.step(1, 5, 0.01)
        x0, v0 = s.state()
        vnew = rng.normal(size=v0.shape)
        s.set_state(vel=vnew)
        x1, v1 = s.state()
        assert np.array_equal(x1, x0) and np.array_equal(v1, vnew)
        # positions outside the box are folded; velocities kept
        xnew = x0 + cfg1.L * rng.integers(-2, 3, size=x0.shape)
        s.set_state(pos=xnew)
        x2, v2 = s.state()
        assert np.array_equal(v2, vnew)
        d = x2 - x0
        assert np.abs(d - cfg1.L * np.rint(d / cfg1.L)).max() < 1e-12
        assert np.all((x2 >= 0) & (x2 < cfg1.L))
        # forces at the new state equal the oracle's
        f2, f3 = s.forces()
    r2, _, _ = oracle.lj_brute(x2, cfg1.L, 1.0, 1.0, 2.5)
    r3, _, _, _ = oracle.atm_brute(x2, cfg1.L, NU, 2.5)
    for got, ref in ((f2, r2), (f3, r3)):
        frms = np.sqrt((ref ** 2).sum(1).mean())
        err = np.linalg.norm(got - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), frms)
        assert err.max() <= 1e-12


def test_non_finite_input_changes_nothing(gpu_lib, cfg1):
    with gpu_lib.System.create(cfg1.x, cfg1.L, cfg1.v, precision=0, nu=NU) as s:
        s.step(1, 5, 0.01)
        x0, v0 = s.state()
        bad = v0.copy()
        bad[17, 2] = np.inf
        with pytest.raises(gpu_lib.MDError) as e:
            s.set_state(x0 * 0.5, bad)
        assert e.value.status == -4
        x1, v1 = s.state()
        assert np.array_equal(x1, x0) and np.array_equal(v1, v0)
        s.step(1, 5, 0.01)  # still usable


def test_runs_are_reproducible_with_the_per_particle_triplet_kernel(gpu_lib, cfg1):
    """The sorted order inside each cell is a function of the positions (Morton key, then index), the
    pair lists are compacted in that order and the per-particle triplet kernel sums each particle's
    force in a fixed order: two runs from the same input agree bit for bit."""
    out = []
    for _ in range(2):
        with gpu_lib.System.create(cfg1.x, cfg1.L, cfg1.v, precision=0, nu=NU, atm_kernel=1) as s:
            s.step(3, 5, 0.01)
            x, v = s.state()
            f2, f3 = s.forces()
        out.append((x, v, f2, f3))
    for a, b in zip(*out):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("classes", [False, True])
def test_runs_are_reproducible_with_the_rotation_triplet_kernel(gpu_lib, cfg1, classes):
    """The rotation kernel (the default FP32 triplet kernel) and the near-class kernel scatter one force
    term per (owner, member) into 64-bit fixed-point sums, whose integer additions give the same result
    in any order: two runs from the same input agree bit for bit, forces and trajectory alike."""
    out = []
    for _ in range(2):
        with gpu_lib.System.create(cfg1.x, cfg1.L, cfg1.v, precision=0, nu=NU, atm_kernel=2) as s:
            if classes:
                s.set_distance_classes(1.5, 5)
            f2a, f3a = s.forces()
            s.step(3, 10, 0.02)
            x, v = s.state()
            f2, f3 = s.forces()
            assert s.stats()["atm_kernel"] == 2
        out.append((f2a, f3a, x, v, f2, f3))
    for a, b in zip(*out):
        assert np.array_equal(a, b)
