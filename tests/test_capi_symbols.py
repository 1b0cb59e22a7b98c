"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/gmls.h (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_2104_14447_gb300 import build, gmls

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    inc = os.path.join(ROOT, "include")
    for fn in sorted(os.listdir(inc)):
        if fn.endswith(".h"):
            text = open(os.path.join(inc, fn)).read()
            names += re.findall(r"^\s*(?:gmls_status|const char\*)\s+(gmls_\w+)\s*\(", text, re.M)
    return names


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert "gmls_stencils" in names and "gmls_assemble_csr" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(gmls.EXPORTED) <= set(names)


def test_binding_loads_and_rejects_bad_arguments_without_gpu():
    build.build()
    L = gmls.load()
    assert b"sm_103a" in L.gmls_version()
    h = ctypes.c_void_p()
    # NULL arena is rejected on the host before any CUDA call
    assert L.gmls_create(ctypes.byref(h), 0, None, None, 1 << 30) == gmls.EINVAL
    assert b"arena" in L.gmls_last_error(None)
