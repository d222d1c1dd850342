"""The C-ABI library builds for sm_103a, loads, and exports every entry point include/voxsim.h
declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "voxsim.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:sim_status|const char\*)\s+(\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2405_00698_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("sim_create", "sim_set_population", "sim_step_n", "sim_fitness", "evo_generation",
                 "sim_backward", "sim_destroy", "sim_last_error"):
        assert name in syms


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_binding_covers_every_export(libpath):
    from paper_2405_00698_gb300 import voxsim
    assert sorted(voxsim.EXPORTS) == sorted(declared_symbols())
