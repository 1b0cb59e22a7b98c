"""The product path and the oracle stay apart (CPU only).

* no module of the package imports the oracle, and importing the binding
  does not load it;
* bench.py imports it only inside the functions of its CPU-baseline and
  reference legs (and the oracle side of its sampled comparisons);
* without the built library, or without a GPU, the binding raises instead
  of computing anything on the host.
"""
import ast
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2104_14447_gb300")

ORACLE_LEGS = {"porous_cpu_baseline", "batched_oracle_errors", "stokes2d_oracle_check", "run_reference"}


def _oracle_imports(tree):
    """(enclosing top-level function or None, line) of every import of the oracle."""
    out = []
    for top in tree.body:
        for node in ast.walk(top):
            names = []
            if isinstance(node, ast.Import):
                names = [a.name for a in node.names]
            elif isinstance(node, ast.ImportFrom):
                names = [node.module or ""]
            if any(n == "oracle" or n.startswith("oracle.") for n in names):
                out.append((top.name if isinstance(top, ast.FunctionDef) else None, node.lineno))
    return out


def test_package_never_imports_the_oracle():
    for dirpath, _, files in os.walk(PKG):
        if "_build" in dirpath:
            continue
        for fn in files:
            if fn.endswith(".py"):
                path = os.path.join(dirpath, fn)
                assert _oracle_imports(ast.parse(open(path).read())) == [], path


def test_binding_import_does_not_load_the_oracle():
    code = ("import sys; import paper_2104_14447_gb300.gmls, paper_2104_14447_gb300.inputs; "
            "assert 'oracle' not in sys.modules")
    subprocess.run([sys.executable, "-c", code], cwd=ROOT, check=True)


def test_bench_uses_the_oracle_only_in_its_cpu_legs():
    found = _oracle_imports(ast.parse(open(os.path.join(ROOT, "bench.py")).read()))
    assert found, "the CPU-baseline leg should time the oracle"
    for fn, line in found:
        assert fn in ORACLE_LEGS, (fn, line)


def test_binding_fails_loudly_without_library(tmp_path):
    code = ("from paper_2104_14447_gb300 import gmls; "
            f"gmls.load({str(tmp_path / 'missing' / 'libgmls.so')!r})")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True)
    assert r.returncode != 0 and "libgmls not built" in r.stderr


def test_context_fails_loudly_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2104_14447_gb300 import build, gmls

    build.build()
    with pytest.raises(Exception):
        gmls.Context(0, arena_bytes=1 << 30)


def test_oracle_shares_no_code_with_the_cuda_path():
    """The oracle's C source includes system headers only, its Python modules
    import nothing from the package, and no native source or build script of
    the package refers to the oracle."""
    import re

    odir = os.path.join(ROOT, "oracle")
    for fn in os.listdir(odir):
        path = os.path.join(odir, fn)
        if fn.endswith((".c", ".h")):
            for inc in re.findall(r'^\s*#\s*include\s*([<"][^>"]+[>"])', open(path).read(), re.M):
                assert inc.startswith("<"), (fn, inc)
        elif fn.endswith(".py"):
            tree = ast.parse(open(path).read())
            for node in ast.walk(tree):
                mods = []
                if isinstance(node, ast.Import):
                    mods = [a.name for a in node.names]
                elif isinstance(node, ast.ImportFrom) and node.level == 0:
                    mods = [node.module or ""]
                assert not any(m.startswith("paper_2104_14447_gb300") for m in mods), (fn, mods)
    csrc = os.path.join(PKG, "csrc")
    for fn in os.listdir(csrc):
        if fn.endswith((".cu", ".cuh", ".h", ".cpp", ".py")):
            assert "oracle" not in open(os.path.join(csrc, fn)).read(), fn
    assert "oracle" not in open(os.path.join(PKG, "build.py")).read()
