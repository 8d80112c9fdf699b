"""The C-ABI library on a machine without a GPU: it builds, loads, and exports
every function that include/iblb.h declares (no compute call is made)."""
import ctypes
import os
import re

from paper_2604_17463_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "iblb.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)       # drop comments
    names = set(re.findall(r"\b(iblb_\w+)\s*\(", text))
    # keep function declarations only (types end in _t / are typedef'd structs)
    return sorted(n for n in names if not n.endswith(("_t", "_s")))


def test_header_declares_the_core_calls():
    names = declared_functions()
    for core in ("iblb_create", "iblb_set_interface", "iblb_step", "iblb_read_fields",
                 "iblb_observables", "iblb_destroy", "iblb_batch_admit", "iblb_inside_mask",
                 "iblb_set_equilibrium", "iblb_deformation", "iblb_mass_static"):
        assert core in names, core


def test_library_exports_every_declared_function():
    lib = ctypes.CDLL(build.build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_are_host_only():
    lib = ctypes.CDLL(build.build())
    lib.iblb_status_string.restype = ctypes.c_char_p
    lib.iblb_status_string.argtypes = [ctypes.c_int]
    assert lib.iblb_status_string(0)
    assert b"classification" in lib.iblb_status_string(8)
