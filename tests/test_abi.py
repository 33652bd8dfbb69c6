"""The C-ABI library builds, loads without a GPU and exports every function of include/kfbi.h."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2309_01068_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_exports_every_declared_function(lib):
    from paper_2309_01068_gb300 import kfbi

    names = kfbi.header_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(kfbi._SIGNATURES), "binding and header disagree"


def test_no_cuda_runtime_dependency(lib):
    from paper_2309_01068_gb300 import build

    out = subprocess.run(["ldd", build.LIB], capture_output=True, text=True).stdout
    assert "libcudart" not in out


def test_status_strings(lib):
    lib.kfbi_status_string.restype = ctypes.c_char_p
    for code in range(10):
        assert lib.kfbi_status_string(code)


def test_header_documents_each_entry_point():
    text = open(os.path.join(ROOT, "include", "kfbi.h")).read()
    for name in re.findall(r"\b(kfbi_\w+)\s*\(", text):
        assert text.count(name) >= 1


def test_no_oracle_import_in_product():
    pkg = os.path.join(ROOT, "paper_2309_01068_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"#.*|//.*", "", src).replace("oracles", ""), f


def test_binding_constants_match_header():
    """Every KFBI_* enumerator the header gives a value has that value in the binding, under
    the same name without the KFBI_ prefix, so the Python side cannot drift from the C side."""
    from paper_2309_01068_gb300 import kfbi

    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "kfbi.h")).read(), flags=re.S)
    pairs = re.findall(r"\bKFBI_([A-Z0-9_]+)\s*=\s*(\d+)", text)
    assert len(pairs) >= 30
    checked = 0
    for name, value in pairs:
        if hasattr(kfbi, name):
            assert getattr(kfbi, name) == int(value), name
            checked += 1
    for name in ("OK", "ERR_ARG", "ERR_CAPACITY", "BOX_FREESPACE_DL", "MIXED", "DOUBLE", "BIE_STEFAN_SL",
                 "OPT_FUSE_INTERP", "OPT_FUSE_DFT", "OPT_BODY_CAP", "OPT_SWEEP_CAP"):
        assert hasattr(kfbi, name), name
    assert checked >= 25
