"""The C-ABI library loads without a GPU and exports every entry point that
include/dynbond.h declares; the binding mirrors the header's structs."""

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1108_4214_gb300 import _build
    try:
        return _build.build()
    except RuntimeError as e:  # no nvcc on this machine
        pytest.skip(str(e))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "dynbond.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dynbond_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("dynbond_create", "dynbond_step", "dynbond_forces", "dynbond_get_topology", "dynbond_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(lib_path)
    for n in declared_functions():
        assert hasattr(lib, n)


def test_binding_matches_header(lib_path):
    from paper_1108_4214_gb300 import dynbond
    assert sorted(dynbond.EXPORTS) == declared_functions()
    L = dynbond.load()
    assert L.dynbond_status_string(3) == b"capacity exceeded"
    assert ctypes.sizeof(dynbond.Rule) == 64
    assert ctypes.sizeof(dynbond.Params) == 64
    assert ctypes.sizeof(dynbond.SystemDesc) == 72
    # bond_k, bond_r0, angle_k, dihedral_k, angle_theta0 (double); dihedral_d, angle_style (int32)
    assert ctypes.sizeof(dynbond.ForceField) == 5 * 16 * 8 + 2 * 16 * 4
    # cell_scale (double); bead / candidate blocks, front_ms, tuned, cell_zdiv, octant (4 bytes each)
    assert ctypes.sizeof(dynbond.Tuning) == 8 + 8 * 4


def test_create_rejects_bad_input_without_touching_the_device(lib_path):
    # malformed rules are rejected during host validation, before any CUDA call
    from paper_1108_4214_gb300 import dynbond
    L = dynbond.load()
    p = dynbond.Params()
    rules = (dynbond.Rule * 1)()
    rules[0].kind = 99
    sd = dynbond.SystemDesc()
    ff = dynbond.ForceField()
    h = ctypes.c_void_p()
    st = L.dynbond_create(ctypes.byref(p), rules, 1, ctypes.byref(sd), ctypes.byref(ff), None, ctypes.byref(h))
    assert st == 1 and not h.value
    assert b"unknown rule kind" in L.dynbond_last_error(None)
