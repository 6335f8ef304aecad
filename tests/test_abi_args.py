"""Argument checks of every C-ABI entry point, without a GPU.

Each call below is rejected by the library's host-side validation before any CUDA call, so these run
on a machine without a device: NULL handles and outputs, invalid sizes, time steps and parameters,
non-finite inputs and capacity limits map to the status codes that include/respa3b.h documents.
"""
import ctypes
import math

import pytest

import paper_2507_11172_gb300 as r3

OK, ARG, BOX, NONFINITE, STATE, CAPACITY = 0, -1, -3, -4, -7, -8


@pytest.fixture(scope="module")
def lib():
    return r3.load()


def _doubles(values):
    return (ctypes.c_double * len(values))(*values)


def test_null_system_handle_is_rejected_everywhere(lib):
    d = ctypes.c_double()
    i64 = ctypes.c_int64()
    i32 = ctypes.c_int()
    buf = _doubles([0.0] * 9)
    counts = (ctypes.c_uint64 * 4)()
    stats = r3.md_stats()
    calls = {
        "md_set_potentials": lambda: lib.md_set_potentials(None, 1.0, 1.0, 2.5, 0.073, 2.5),
        "md_set_skin": lambda: lib.md_set_skin(None, 0.3),
        "md_set_distance_classes": lambda: lib.md_set_distance_classes(None, 1.5, 2),
        "md_get_near_forces": lambda: lib.md_get_near_forces(None, buf),
        "md_respa_step": lambda: lib.md_respa_step(None, 1, 1, 0.01),
        "md_get_forces": lambda: lib.md_get_forces(None, buf, buf),
        "md_get_energy": lambda: lib.md_get_energy(None, ctypes.byref(d), ctypes.byref(d), ctypes.byref(d),
                                                   ctypes.byref(d)),
        "md_get_rdf": lambda: lib.md_get_rdf(None, 4, 2.0, counts),
        "md_get_state": lambda: lib.md_get_state(None, buf, buf),
        "md_set_state": lambda: lib.md_set_state(None, buf, buf),
        "md_get_stats": lambda: lib.md_get_stats(None, ctypes.byref(stats)),
        "md_set_profiling": lambda: lib.md_set_profiling(None, 1),
        "md_set_atm_kernel": lambda: lib.md_set_atm_kernel(None, 2),
        "md_set_lj_kernel": lambda: lib.md_set_lj_kernel(None, 1),
        "md_inject_copy_shortfall": lambda: lib.md_inject_copy_shortfall(None, 16),
        "md_get_info": lambda: lib.md_get_info(None, ctypes.byref(i64), ctypes.byref(d), ctypes.byref(i32)),
        "md_get_memory": lambda: lib.md_get_memory(None, ctypes.byref(ctypes.c_size_t())),
        "md_set_shapes": lambda: lib.md_set_shapes(None, 64, 4, 8),
    }
    for name, call in calls.items():
        assert call() == ARG, name
    assert lib.md_destroy_system(None) == OK  # NULL-safe


def test_null_batch_handle_is_rejected_everywhere(lib):
    u = ctypes.c_uint64()
    i32 = ctypes.c_int()
    d = ctypes.c_double()
    assert lib.md_batch_create(None, 1 << 30) == ARG
    assert lib.md_batch_submit(None, None, 1, 1, 0.01, ctypes.byref(u)) == ARG
    assert lib.md_batch_run(None, 0) == ARG
    assert lib.md_batch_poll(None, 0, ctypes.byref(i32)) == ARG
    assert lib.md_batch_latency(None, 0, ctypes.byref(d), ctypes.byref(i32)) == ARG
    assert lib.md_batch_pending(None, ctypes.byref(i32), ctypes.byref(i32)) == ARG
    assert lib.md_batch_cycles(None, ctypes.byref(u), ctypes.byref(u)) == ARG
    assert lib.md_batch_cancel(None, 1) == ARG
    assert lib.md_batch_set_limits(None, 1000) == ARG
    assert lib.md_batch_destroy(None) == OK  # NULL-safe


def test_create_system_validation_before_any_device_work(lib):
    h = ctypes.c_void_p()
    n = 4
    pos = _doubles([0.5 * q for q in range(3 * n)])
    assert lib.md_create_system(None, n, 20.0, pos, None, 1.0, 0, None) == ARG       # no output handle
    assert lib.md_create_system(ctypes.byref(h), n, 20.0, None, None, 1.0, 0, None) == ARG  # no positions
    assert lib.md_create_system(ctypes.byref(h), n, 0.0, pos, None, 1.0, 0, None) == ARG    # box length 0
    assert lib.md_create_system(ctypes.byref(h), n, math.nan, pos, None, 1.0, 0, None) == ARG
    assert lib.md_create_system(ctypes.byref(h), n, math.inf, pos, None, 1.0, 0, None) == ARG  # infinite box
    assert lib.md_create_system(ctypes.byref(h), n, 20.0, pos, None, 0.0, 0, None) == ARG   # mass 0
    assert lib.md_create_system(ctypes.byref(h), n, 20.0, pos, None, math.inf, 0, None) == ARG  # infinite mass
    assert lib.md_create_system(ctypes.byref(h), n, 20.0, pos, None, math.nan, 0, None) == ARG
    assert lib.md_create_system(ctypes.byref(h), n, 20.0, pos, None, 1.0, 7, None) == ARG   # precision
    bad = _doubles([0.5 * q for q in range(3 * n)])
    bad[4] = math.inf
    assert lib.md_create_system(ctypes.byref(h), n, 20.0, bad, None, 1.0, 0, None) == NONFINITE
    vel = _doubles([0.0] * (3 * n))
    vel[7] = math.nan
    assert lib.md_create_system(ctypes.byref(h), n, 20.0, pos, vel, 1.0, 0, None) == NONFINITE
    # L must exceed 3 r_c (default r_c2 = r_c3 = 2.5): 7.0 is too small even with the skin thinned to 0
    assert lib.md_create_system(ctypes.byref(h), n, 7.0, pos, None, 1.0, 0, None) == BOX
    assert not h.value  # nothing was created


def test_direct_sum_validation_before_any_device_work(lib):
    n = 5
    pos = _doubles([0.7 * q for q in range(3 * n)])
    f3 = _doubles([0.0] * (3 * n))
    u3 = ctypes.c_double()
    assert lib.md_atm_direct(None, n, 0.073, 0, f3, ctypes.byref(u3), None) == ARG
    assert lib.md_atm_direct(pos, n, 0.073, 0, None, ctypes.byref(u3), None) == ARG
    assert lib.md_atm_direct(pos, 2, 0.073, 0, f3, ctypes.byref(u3), None) == ARG       # n < 3
    assert lib.md_atm_direct(pos, n, -1.0, 0, f3, ctypes.byref(u3), None) == ARG        # nu < 0
    assert lib.md_atm_direct(pos, n, math.nan, 0, f3, ctypes.byref(u3), None) == ARG
    assert lib.md_atm_direct(pos, n, 0.073, 3, f3, ctypes.byref(u3), None) == ARG       # precision
    bad = _doubles([0.7 * q for q in range(3 * n)])
    bad[2] = math.nan
    assert lib.md_atm_direct(bad, n, 0.073, 0, f3, ctypes.byref(u3), None) == NONFINITE
    # the whole system is staged in one CTA's shared memory: larger n is a capacity error
    big = 20000
    posb = _doubles([0.0] * (3 * big))
    fb = _doubles([0.0] * (3 * big))
    assert lib.md_atm_direct(posb, big, 0.073, 0, fb, ctypes.byref(u3), None) == CAPACITY


def test_noalloc_validation_before_any_device_work(lib):
    # pointers are only checked for NULL before the device set-up; host buffers stand in here and are
    # never dereferenced on these paths
    n = 8
    pos = _doubles([0.0] * (3 * n))
    f3 = _doubles([0.0] * (3 * n))
    u3 = ctypes.c_double()
    trip = ctypes.c_uint64()
    call = lib.md_atm_forces_noalloc
    assert call(None, n, 20.0, 0.073, 2.5, f3, ctypes.byref(u3), ctypes.byref(trip), None) == ARG
    assert call(pos, n, 20.0, 0.073, 2.5, None, ctypes.byref(u3), ctypes.byref(trip), None) == ARG
    assert call(pos, 2, 20.0, 0.073, 2.5, f3, ctypes.byref(u3), ctypes.byref(trip), None) == ARG
    assert call(pos, n, 20.0, 0.073, 0.0, f3, ctypes.byref(u3), ctypes.byref(trip), None) == ARG
    assert call(pos, n, 20.0, -0.5, 2.5, f3, ctypes.byref(u3), ctypes.byref(trip), None) == ARG
    assert call(pos, n, 7.5, 0.073, 2.5, f3, ctypes.byref(u3), ctypes.byref(trip), None) == BOX  # L = 3 r_c
    assert call(pos, n, math.inf, 0.073, 2.5, f3, ctypes.byref(u3), ctypes.byref(trip), None) == ARG
    assert call(pos, n, math.nan, 0.073, 2.5, f3, ctypes.byref(u3), ctypes.byref(trip), None) == ARG
    assert call(pos, n, 20.0, 0.073, math.inf, f3, ctypes.byref(u3), ctypes.byref(trip), None) == ARG
    assert call(pos, n, 20.0, math.inf, 2.5, f3, ctypes.byref(u3), ctypes.byref(trip), None) == ARG
    big = 16385  # MD_NOALLOC_MAX_N + 1
    assert call(pos, big, 100.0, 0.073, 2.5, f3, ctypes.byref(u3), ctypes.byref(trip), None) == CAPACITY
    # the rejection's message is the one md_last_error returns
    assert b"MD_NOALLOC_MAX_N" in lib.md_last_error()


def test_status_strings_cover_every_code(lib):
    seen = set()
    for code in (OK, ARG, -2, BOX, NONFINITE, -5, -6, STATE, CAPACITY, -9):
        s = lib.md_status_string(code)
        assert s and isinstance(s, bytes)
        seen.add(s)
    assert len(seen) == 10  # distinct texts


def test_peak_measurement_validation_before_any_device_work(lib):
    f = ctypes.c_double()
    assert lib.md_measure_fma_peak(3, 10.0, ctypes.byref(f), None) == ARG   # unknown kind
    assert lib.md_measure_fma_peak(-1, 10.0, ctypes.byref(f), None) == ARG
    assert lib.md_measure_fma_peak(0, 10.0, None, None) == ARG                # no output
    assert lib.md_measure_fma_peak(0, 0.0, ctypes.byref(f), None) == ARG     # duration
    assert lib.md_measure_fma_peak(0, math.nan, ctypes.byref(f), None) == ARG
