"""The oracle and the CUDA path share no code, and the product path cannot reach the
oracle: no module or source file of the package names the oracle, no source of the oracle
names the package's sources, and the library the package builds is compiled from the
package's own sources only.  The seeded input generators (workloads.py) hold no
arithmetic of the method: they import nothing from either side."""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2403_04267_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _files(top, exts):
    for d, _, fs in os.walk(top):
        if "_build" in d or "__pycache__" in d:
            continue
        for f in fs:
            if f.endswith(exts):
                yield os.path.join(d, f)


def _imports(path):
    tree = ast.parse(open(path).read())
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            for a in node.names:
                yield a.name
        elif isinstance(node, ast.ImportFrom):
            yield (node.module or "") if node.level == 0 else "." + (node.module or "")


def test_package_never_imports_or_includes_the_oracle():
    for path in _files(PKG, (".py",)):
        for mod in _imports(path):
            assert not mod.split(".")[0] == "oracle", (path, mod)
    for path in _files(PKG, (".cu", ".cuh", ".h", ".c", ".cpp")):
        src = open(path).read()
        assert not re.search(r'#include\s+"[^"]*oracle', src), path
    for path in _files(os.path.join(ROOT, "include"), (".h",)):
        assert "oracle" not in open(path).read().lower(), path


def test_oracle_never_uses_the_package_sources():
    for path in _files(ORACLE, (".py",)):
        for mod in _imports(path):
            assert not mod.startswith("paper_2403_04267_gb300.csrc"), (path, mod)
            assert mod not in ("paper_2403_04267_gb300.salec", "paper_2403_04267_gb300.surrogate",
                               "paper_2403_04267_gb300.build"), (path, mod)
    for path in _files(ORACLE, (".c", ".h")):
        src = open(path).read()
        assert not re.search(r'#include\s+"[^"]*(salec_|mlp_)', src), path


def test_input_generators_hold_no_code_of_either_side():
    path = os.path.join(PKG, "workloads.py")
    for mod in _imports(path):
        top = mod.split(".")[0]
        assert top in ("__future__", "math", "numpy", "copy", "typing", "dataclasses", ""), (path, mod)


def test_library_sources_are_the_package_own():
    from paper_2403_04267_gb300 import build as B
    for src in B.SOURCES:
        assert os.path.exists(os.path.join(PKG, "csrc", src)), src
        assert "oracle" not in src
