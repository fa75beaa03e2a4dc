"""The oracle and the CUDA path share no code (CPU only): the oracle's C file
includes only system headers and its Python side imports nothing from the
package; the package (kernels, binding, build, generators) never includes,
imports or calls the oracle; the benchmark imports it only inside its CPU
legs, never at module level."""
import ast
import os
import re
from pathlib import Path

ROOT = Path(__file__).resolve().parent.parent
PKG = ROOT / "paper_1608_02148_gb300"


def test_oracle_uses_no_project_code():
    c = (ROOT / "oracle" / "rsvd_oracle.c").read_text()
    assert not re.findall(r'#include\s+"', c)
    tree = ast.parse((ROOT / "oracle" / "__init__.py").read_text())
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            assert all(not a.name.startswith("paper_1608_02148_gb300") for a in node.names)
        elif isinstance(node, ast.ImportFrom):
            assert not (node.module or "").startswith("paper_1608_02148_gb300")


def test_package_never_touches_the_oracle():
    for f in list((PKG / "csrc").glob("*.cu")) + list((PKG / "csrc").glob("*.cuh")) + list((ROOT / "include").glob("*.h")):
        text = f.read_text()
        assert not re.search(r'#include\s+"[^"]*oracle', text), f.name
        assert "oracle_" not in text, f.name  # no oracle symbol referenced
    for f in PKG.glob("*.py"):
        tree = ast.parse(f.read_text())
        for node in ast.walk(tree):
            if isinstance(node, ast.Import):
                assert all(a.name.split(".")[0] != "oracle" for a in node.names), f.name
            elif isinstance(node, ast.ImportFrom):
                assert (node.module or "").split(".")[0] != "oracle", f.name


def test_bench_imports_the_oracle_only_inside_functions():
    tree = ast.parse((ROOT / "bench.py").read_text())
    for node in tree.body:  # module level
        if isinstance(node, ast.Import):
            assert all(a.name.split(".")[0] != "oracle" for a in node.names)
        elif isinstance(node, ast.ImportFrom):
            assert (node.module or "").split(".")[0] != "oracle"
