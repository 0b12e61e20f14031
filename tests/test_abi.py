"""The C ABI: the library builds for sm_103a, loads, exports every symbol include/drot.h
declares, and the ctypes structs match the C layouts.  No compute call is made (no GPU here)."""

import ctypes
import os
import re
import subprocess

import pytest

from paper_2110_11738_b300 import build as libbuild
from paper_2110_11738_b300 import drot

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "drot.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(drot_[a-z0-9_]+)\s*\(", text)))


def test_library_builds_and_exports_every_declared_symbol():
    path = libbuild.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    declared = _declared_functions()
    assert set(declared) == set(drot.EXPORTED)
    for name in declared:
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (drot_[a-z0-9_]+)$", out, flags=re.M))
    assert set(declared) <= exported


def test_status_strings_without_gpu():
    lib = drot.load()
    for code in range(9):  # DROT_OK .. DROT_ERR_TOO_LARGE
        assert lib.drot_status_string(code)
    assert lib.drot_status_string(5) == b"iteration cap reached"
    assert b"static workspace" in lib.drot_status_string(drot.DROT_ERR_TOO_LARGE)


def test_ctypes_layouts_match_c(tmp_path):
    src = tmp_path / "sizes.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "drot.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu\\n\", sizeof(drot_config), sizeof(drot_result),"
        " sizeof(drot_problem), sizeof(drot_profile), offsetof(drot_result, status), offsetof(drot_config, profile));"
        "return 0;}\n")
    exe = tmp_path / "sizes"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    vals = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert vals == [ctypes.sizeof(drot.DrotConfig), ctypes.sizeof(drot.DrotResult),
                    ctypes.sizeof(drot.DrotProblem), ctypes.sizeof(drot.DrotProfile),
                    drot.DrotResult.status.offset, drot.DrotConfig.profile.offset]


def test_create_without_device_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = drot.load()
    h = ctypes.c_void_p()
    st = lib.drot_create(ctypes.byref(h), None)
    assert st == drot.DROT_ERR_CUDA and not h.value
    assert lib.drot_destroy(None) == 0


def _static_call(lib, m, n, ld, C=16, p=8, q=8, X=16, mu=8, nu=8, tol=1e-6, max_iter=10):
    # The pointer values are never dereferenced: every case below is refused by the host-side
    # checks before the library asks the driver for the current device.
    return lib.drot_solve_static(m, n, C, ld, p, q, 0.0, tol, max_iter, X, mu, nu, 0, None, None)


@pytest.mark.parametrize("case", [
    dict(m=0, n=4, ld=4),                   # empty: no source points
    dict(m=4, n=0, ld=4),                   # empty: no target points
    dict(m=-3, n=4, ld=4),
    dict(m=4, n=5, ld=4),                   # pitch shorter than a row
    dict(m=4, n=5, ld=6),                   # pitch not a multiple of 4 floats (16-byte rows)
    dict(m=4, n=4, ld=4, C=0),              # NULL buffers
    dict(m=4, n=4, ld=4, nu=0),
    dict(m=4, n=4, ld=4, X=24),             # X not 16-byte aligned
    dict(m=4, n=4, ld=4, p=12),             # p not 8-byte aligned
    dict(m=4, n=4, ld=4, max_iter=-1),
    dict(m=4, n=4, ld=4, tol=float("nan")),
    dict(m=1 << 30, n=1 << 12, ld=1 << 12),  # m * n beyond 2^40 entries
])
def test_static_solve_rejects_bad_arguments_without_touching_the_device(case):
    lib = drot.load()
    assert _static_call(lib, **case) == drot.DROT_ERR_INVALID_ARG


def test_handle_calls_reject_a_null_handle():
    lib = drot.load()
    res = drot.DrotResult()
    assert lib.drot_solve(None, 4, 4, 16, 4, 8, 8, 0.0, 1e-6, 10, 16, 8, 8, 0, ctypes.byref(res)) == \
        drot.DROT_ERR_INVALID_ARG
    assert lib.drot_solve_f64(None, 4, 4, 16, 4, 8, 8, 0.0, 1e-6, 10, 16, 8, 8, 0, ctypes.byref(res)) == \
        drot.DROT_ERR_INVALID_ARG
    assert lib.drot_solve_batched(None, 1, None, 1e-6, 10, 0, None) == drot.DROT_ERR_INVALID_ARG
    assert lib.drot_get_profile(None, ctypes.byref(drot.DrotProfile())) == drot.DROT_ERR_INVALID_ARG
    assert lib.drot_reset_profile(None) == drot.DROT_ERR_INVALID_ARG
    assert lib.drot_last_error(None) == b""
