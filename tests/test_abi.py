"""CPU-side checks of the C ABI: the library builds, loads, and exports every
function that include/tc.h declares (no GPU call is made)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1804_06926_gb300 import _build, binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "tc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(tc_[a-z_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_expected_entry_points():
    names = declared_functions()
    for required in ("tc_build_oriented_csr", "tc_count", "tc_count_batch", "tc_submit", "tc_poll"):
        assert required in names


def test_library_exports_every_declared_symbol():
    path = _build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (tc_[a-z_]+)\b", out))
    assert set(declared_functions()) <= exported
    # the Python binding covers the same names
    assert set(binding.EXPORTS) == set(declared_functions())


def test_header_compiles_as_c():
    src = '#include "tc.h"\nint main(void){ tc_config c = {0}; (void)c; return 0; }\n'
    r = subprocess.run(["gcc", "-x", "c", "-std=c99", "-fsyntax-only", "-I", os.path.join(ROOT, "include"), "-"],
                       input=src, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
