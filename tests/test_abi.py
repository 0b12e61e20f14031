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
    for code in range(8):
        assert lib.drot_status_string(code)
    assert lib.drot_status_string(5) == b"iteration cap reached"


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
