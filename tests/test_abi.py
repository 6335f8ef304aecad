"""The C-ABI library loads and exports every entry point declared in include/respa3b.h.

Runs without a GPU: only symbol lookup, the pure status-string function and
argument checks that return before any CUDA call.
"""
import ctypes
import os
import re

import pytest

import paper_2507_11172_gb300 as r3

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "respa3b.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(md_[a-z_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("md_create_system", "md_set_potentials", "md_respa_step", "md_get_forces", "md_get_energy",
                 "md_get_state", "md_set_state", "md_destroy_system", "md_batch_create", "md_batch_submit",
                 "md_batch_run", "md_batch_poll"):
        assert must in names


def test_library_exports_every_declared_symbol():
    r3.build_lib.build()
    lib = ctypes.CDLL(r3.library_path())
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in r3.SIGNATURES, name


def test_status_strings_and_argument_checks_without_gpu():
    lib = r3.load()
    assert lib.md_status_string(0) == b"ok"
    assert b"box" in lib.md_status_string(-3)
    h = ctypes.c_void_p()
    pos = (ctypes.c_double * 6)()
    # n < 3 and a box not larger than 3 r_c are rejected before any device work
    assert lib.md_create_system(ctypes.byref(h), 2, 20.0, pos, None, 1.0, 0, None) == -1
    pos9 = (ctypes.c_double * 9)()
    assert lib.md_create_system(ctypes.byref(h), 3, 5.0, pos9, None, 1.0, 0, None) == -3
    assert lib.md_destroy_system(None) == 0
    assert lib.md_respa_step(None, 1, 1, 0.01) == -1


def test_no_oracle_import_in_product_package():
    pkg = os.path.join(ROOT, "paper_2507_11172_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "liboracle" not in src and "oracle/" not in src, f


def test_binding_argument_counts_match_the_header():
    """Every ctypes signature of the binding has as many arguments as the header's prototype."""
    txt = open(os.path.join(ROOT, "include", "respa3b.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    protos = dict(re.findall(r"\b(md_[a-z_]+)\s*\(([^)]*)\)\s*;", txt))
    assert protos
    for name, params in protos.items():
        params = params.strip()
        n = 0 if params in ("", "void") else params.count(",") + 1
        assert len(r3.SIGNATURES[name][1]) == n, name
