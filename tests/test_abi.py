"""CPU checks of the C-ABI library: it builds, loads without a GPU, exports
every entry point include/tc.h declares, does not link the oracle, and
rejects bad arguments before touching the device."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1910_02371_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    src = open(os.path.join(ROOT, "include", "tc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tc_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_hot_path():
    names = declared_functions()
    for n in ["tc_build_pattern", "tc_tttp", "tc_mttkrp", "tc_solve_factor", "tc_loss_grad",
              "tc_ggn_matvec", "tc_cg_solve", "tc_ggn_step", "tc_last_error"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_library_does_not_contain_the_oracle():
    from paper_1910_02371_gb300 import build
    out = subprocess.run(["nm", "-D", "--defined-only", build.OUT], capture_output=True, text=True).stdout
    assert "orc_" not in out
    assert "tc_tttp" in out


def test_argument_errors_without_device(lib):
    P = ctypes.c_void_p
    lib.tc_build_pattern.argtypes = [ctypes.c_int, P, ctypes.c_int64, P, P, ctypes.c_int,
                                     ctypes.c_uint, P, P]
    out = ctypes.c_void_p()
    dims = (ctypes.c_int64 * 3)(4, 5, 6)
    # order 2 is a valid request this build does not implement
    assert lib.tc_build_pattern(2, dims, 0, None, None, 0, 0, None, ctypes.byref(out)) == 9
    assert lib.tc_build_pattern(3, dims, -1, None, None, 0, 0, None, ctypes.byref(out)) == 1
    assert lib.tc_build_pattern(3, dims, 10, None, None, 0, 0, None, ctypes.byref(out)) == 1
    assert lib.tc_build_pattern(3, dims, 0, None, None, 7, 0, None, ctypes.byref(out)) == 1
    assert lib.tc_build_pattern(3, dims, 0, None, None, 0, 0, None, None) == 1
    # flags: unknown bits, consuming the input without a lean build, lean with
    # the refill work space or the duplicate check
    for flags in (16, 8, 4 | 2, 4 | 1):
        assert lib.tc_build_pattern(3, dims, 0, None, None, 0, flags, None, ctypes.byref(out)) == 1
    bad = (ctypes.c_int64 * 3)(4, 0, 6)
    assert lib.tc_build_pattern(3, bad, 0, None, None, 0, 0, None, ctypes.byref(out)) == 1
    lib.tc_tttp.argtypes = [P, ctypes.c_int, P, ctypes.c_int, P, P, P]
    assert lib.tc_tttp(None, 0, None, 4, None, None, None) == 1
    lib.tc_status_string.restype = ctypes.c_char_p
    assert lib.tc_status_string(6) == b"row system not positive definite"
    lib.tc_launch_count.restype = ctypes.c_int64
    assert lib.tc_launch_count() == 0


def test_python_binding_imports_without_gpu():
    from paper_1910_02371_gb300 import tc
    assert tc.LOSSES["poisson_log"] == 1
    assert callable(tc.tttp) and callable(tc.solve_factor)
