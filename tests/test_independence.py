"""The oracle and the GPU path share no code, and only the tests, smoke() and
bench.py's CPU baseline touch the oracle: a static check of the sources."""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1307_2666_gb300")


def _files(d, exts):
    for dirpath, _, names in os.walk(d):
        if "__pycache__" in dirpath or "_lib" in dirpath:
            continue
        for n in names:
            if n.endswith(exts):
                yield os.path.join(dirpath, n)


def _imports(path):
    tree = ast.parse(open(path).read())
    out = []
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out += [(a.name, node) for a in node.names]
        elif isinstance(node, ast.ImportFrom) and node.module:
            out.append((node.module, node))
    return tree, out


def test_product_package_never_imports_the_oracle():
    for f in _files(PKG, (".py",)):
        _, imps = _imports(f)
        assert not [m for m, _ in imps if m == "oracle" or m.startswith("oracle.")], f
    for f in _files(os.path.join(PKG, "csrc"), (".cpp", ".cu", ".h", ".cuh")):
        assert not re.search(r"#include\s+\"[^\"]*oracle", open(f).read()), f


def test_oracle_never_imports_the_product():
    for f in _files(os.path.join(ROOT, "oracle"), (".py",)):
        _, imps = _imports(f)
        assert not [m for m, _ in imps if m.startswith("paper_1307_2666_gb300")], f


def test_input_generators_import_neither():
    for f in _files(os.path.join(ROOT, "hif_inputs"), (".py",)):
        _, imps = _imports(f)
        assert not [m for m, _ in imps if m.startswith(("oracle", "paper_1307_2666_gb300"))], f


def test_bench_touches_the_oracle_only_in_its_cpu_baseline():
    tree, imps = _imports(os.path.join(ROOT, "bench.py"))
    allowed = {"oracle_sample"}                       # the bounded oracle run (CPU baseline / reference arm)
    owners = {}
    for fn in ast.walk(tree):
        if isinstance(fn, ast.FunctionDef):
            for node in ast.walk(fn):
                owners.setdefault(id(node), fn.name)
    for m, node in imps:
        if m == "oracle" or m.startswith("oracle."):
            assert owners.get(id(node)) in allowed, (m, owners.get(id(node)))
