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


def _header_constants():
    """NAME -> value of every enumerator and #define constant in include/tc.h."""
    src = open(os.path.join(ROOT, "include", "tc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    vals = {}
    for name, v in re.findall(r"\b(TC_[A-Z0-9_]+)\s*=\s*(0x[0-9a-fA-F]+|\d+)", src):
        vals[name] = int(v, 0)
    for name, v in re.findall(r"#define\s+(TC_[A-Z0-9_]+)\s+(0x[0-9a-fA-F]+|\d+)u?\b", src):
        vals[name] = int(v, 0)
    return vals


def test_binding_constants_match_the_header():
    """The Python binding's status codes, dtypes, losses, weight kinds,
    precision forms, pattern flags and Gram engines are the header's values,
    and its tuning struct has the C layout."""
    import ctypes as ct
    from paper_1910_02371_gb300 import tc
    h = _header_constants()
    status = ["OK", "ERR_ARG", "ERR_RANGE", "ERR_DUPLICATE", "ERR_OOM", "ERR_CUDA", "ERR_NOT_SPD",
              "ERR_DOMAIN", "ERR_BREAKDOWN", "ERR_UNSUPPORTED", "ERR_TIMEOUT"]
    for name in status:
        assert getattr(tc, name) == h["TC_" + name], name
    assert (tc.F32, tc.F64) == (h["TC_F32"], h["TC_F64"])
    assert tc.LOSSES == {"ls": h["TC_LOSS_LS"], "poisson_log": h["TC_LOSS_POISSON_LOG"],
                         "poisson_id": h["TC_LOSS_POISSON_ID"]}
    assert (tc.W_ONE, tc.W_VALUES, tc.W_ARRAY) == (h["TC_W_ONE"], h["TC_W_VALUES"], h["TC_W_ARRAY"])
    forms = {"fp32": "TC_PREC_FP32", "tf32_refine": "TC_PREC_TF32_REFINE",
             "bf16_refine": "TC_PREC_BF16_REFINE", "fp32_refine": "TC_PREC_FP32_REFINE"}
    for k, name in forms.items():
        assert tc.PRECS[k] == h[name]
        if k != "fp32":
            assert tc.PRECS[k + "2"] == h[name] | h["TC_PREC_REFINE2"]
            assert tc.PRECS[k + "_chol32"] == h[name] | h["TC_PREC_CHOL32"]
    assert (tc.CHECK_DUPLICATES, tc.REFILLABLE, tc.LEAN, tc.CONSUME_INPUT) == (
        h["TC_PATTERN_CHECK_DUPLICATES"], h["TC_PATTERN_REFILLABLE"], h["TC_PATTERN_LEAN"],
        h["TC_PATTERN_CONSUME_INPUT"])
    assert (tc.GRAM_AUTO, tc.GRAM_WARP_MMA, tc.GRAM_TCGEN05) == (
        h["TC_GRAM_AUTO"], h["TC_GRAM_WARP_MMA"], h["TC_GRAM_TCGEN05"])
    # int64 chunk_nnz, int64 batch_bytes, int32 chol_rows_per_warp, int32 gram_kernel
    assert ct.sizeof(tc._SolveTuning) == 24
    assert [f[0] for f in tc._SolveTuning._fields_] == ["chunk_nnz", "batch_bytes",
                                                       "chol_rows_per_warp", "gram_kernel"]


def test_als_update_rejects_bad_arguments_without_device(lib):
    P = ctypes.c_void_p
    lib.tc_als_update.argtypes = [P, ctypes.c_int, P, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                  P, P, P]
    out = ctypes.c_float(0.0)
    # no pattern
    assert lib.tc_als_update(None, 16, None, 0, 0.5, 0, ctypes.byref(out), None, None) == 1
