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


def test_binding_structs_match_the_header(tmp_path):
    """Every parameter struct of include/gmls.h has the size and field offsets
    of its ctypes mirror in the binding (compiled as C with the host gcc and
    printed; a field added on one side only changes the size or an offset)."""
    import shutil
    import subprocess

    if shutil.which("gcc") is None:
        pytest.skip("no host C compiler")
    structs = {"gmls_nbr_params": gmls.NbrParams, "gmls_stencil_params": gmls.StencilParams,
               "gmls_request": gmls.Request, "gmls_stokes_params": gmls.StokesParams,
               "gmls_gmres_params": gmls.GmresParams, "gmls_serve_stats": gmls.ServerStats}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "gmls.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        s, f, v = ln.split()
        got[(s, f)] = int(v)
    for cname, cls in structs.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)
