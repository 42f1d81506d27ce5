"""The oracle and the CUDA path share no code.

`oracle/` may import only the standard library, numpy/scipy, its own modules
and the seeded input generators; the product package imports nothing from
`oracle/` (or from the benchmark or the tests), and its CUDA sources and
headers do not include anything outside the package and `include/`; the
generators hold no method arithmetic and import only numpy.
"""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = "paper_2511_21640_gb300"


def _imports(path):
    with open(path) as fh:
        tree = ast.parse(fh.read(), filename=path)
    out = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out |= {a.name.split(".")[0] for a in node.names}
        elif isinstance(node, ast.ImportFrom):
            out.add("." if node.level else node.module.split(".")[0])
    return out


def _py_files(d):
    return [os.path.join(ROOT, d, f) for f in sorted(os.listdir(os.path.join(ROOT, d))) if f.endswith(".py")]


def test_oracle_imports_no_product_code():
    allowed = {"__future__", "numpy", "scipy", "math", "itertools", "functools", "re", "collections", ".",
               "oracle", "synthetic"}
    for f in _py_files("oracle"):
        extra = _imports(f) - allowed
        assert not extra, (f, extra)


def test_product_imports_no_oracle():
    forbidden = {"oracle", "bench", "tests", "conftest", "synthetic"}
    for f in _py_files(PKG):
        bad = _imports(f) & forbidden
        assert not bad, (f, bad)


def test_cuda_sources_include_only_the_package_and_the_public_headers():
    csrc = os.path.join(ROOT, PKG, "csrc")
    local = set(os.listdir(csrc))
    public = {os.path.join("..", "..", "include", h) for h in os.listdir(os.path.join(ROOT, "include"))}
    for f in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, f)) as fh:
            for inc in re.findall(r'#include\s+"([^"]+)"', fh.read()):
                assert inc in local or inc in public, (f, inc)


def test_generators_import_only_numpy():
    assert _imports(os.path.join(ROOT, "synthetic", "__init__.py")) <= {"__future__", "numpy"}


def test_binding_fails_loudly_without_the_library(tmp_path):
    """No CPU fallback: the binding, copied without its compiled library,
    refuses to import."""
    import shutil
    import subprocess
    import sys
    pkg = tmp_path / PKG
    pkg.mkdir()
    shutil.copy(os.path.join(ROOT, PKG, "__init__.py"), pkg / "__init__.py")
    out = subprocess.run([sys.executable, "-c", f"import {PKG}"], cwd=tmp_path, capture_output=True, text=True,
                         env={**os.environ, "PYTHONPATH": str(tmp_path)}, timeout=300)
    assert out.returncode != 0
    assert "ImportError" in out.stderr and "libadc_gb300.so is missing" in out.stderr
