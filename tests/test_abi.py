"""CPU checks of the C ABI boundary: the library builds for sm_103a, loads
without a GPU, and exports every entry point that include/dgs.h declares."""
import ctypes
import os
import re

import pytest

from paper_1106_5694_gb300 import binding, build_ext

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dgs.h")


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"DGS_API[^;(]*?\b(dgs_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    path = build_ext.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = _declared()
    for required in ("dgs_solve", "dgs_solve_ex", "dgs_evaluate", "dgs_greedy_init", "dgs_status_string"):
        assert required in names
    assert sorted(binding.EXPORTED) == names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), f"{name} declared in dgs.h but not exported"


def test_status_strings_without_gpu(lib):
    lib.dgs_status_string.restype = ctypes.c_char_p
    lib.dgs_status_string.argtypes = [ctypes.c_int]
    assert lib.dgs_status_string(0) == b"DGS_OK"
    assert lib.dgs_status_string(2) == b"DGS_ERR_RANGE"
    assert lib.dgs_status_string(5) == b"DGS_TIMEOUT"


def test_default_options_without_gpu(lib):
    o = binding.dgs_options()
    o.init = 99
    o.max_sweeps = 7
    lib.dgs_default_options(ctypes.byref(o))
    assert o.init == binding.DGS_INIT_GREEDY and o.max_sweeps == 0 and o.deadline_us == 0


def test_invalid_arguments_rejected_before_any_device_call(lib):
    lib.dgs_solve.restype = ctypes.c_int
    f = ctypes.c_int64(0)
    assert lib.dgs_solve(None, 10, None, ctypes.byref(f), None) == binding.DGS_ERR_INVALID
    assert lib.dgs_solve(ctypes.c_void_p(16), 0, ctypes.c_void_p(16), ctypes.byref(f), None) == binding.DGS_ERR_INVALID


def test_build_targets_sm103a_only():
    assert build_ext.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
