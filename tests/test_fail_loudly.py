"""The product path has no CPU fallback: without its library or without a CUDA device it raises.

Runs on a machine without a GPU (skipped where a device is present, since there the calls succeed).
"""
import numpy as np
import pytest

import paper_2507_11172_gb300 as r3
from md_inputs import fcc_jitter

torch = pytest.importorskip("torch")
no_device = pytest.mark.skipif(torch.cuda.is_available(), reason="a CUDA device is present")


def test_missing_library_raises(monkeypatch, tmp_path):
    monkeypatch.setattr(r3, "_lib", None)
    monkeypatch.setattr(r3.build_lib, "LIB", str(tmp_path / "librespa3b.so"))
    with pytest.raises(RuntimeError, match="missing"):
        r3.load(build_if_missing=False)


@no_device
def test_system_creation_without_a_device_raises():
    x, L = fcc_jitter(1000, 0.8, 0.05, seed=3)  # L = 10.77 > 3 (r_c + skin)
    with pytest.raises(r3.MDError) as e:
        r3.md_create_system(x, L)
    assert e.value.status == -6  # MD_ERR_CUDA: the CUDA runtime call failed, nothing computed on the host


@no_device
def test_direct_sum_without_a_device_raises():
    rng = np.random.default_rng(5)
    x = rng.uniform(0.0, 4.0, size=(20, 3))
    with pytest.raises(r3.MDError) as e:
        r3.md_atm_direct(x, 0.073)
    assert e.value.status in (-2, -6)  # device allocation or runtime failure, never a host result
