"""The oracle and the CUDA path share no code: nothing under oracle/ imports
the product package, and the product package (Python and CUDA sources)
neither imports nor includes anything from oracle/.  The seeded input
generators in scenegen.py are the one module both sides use, and it holds
no arithmetic of the method (it imports only the standard library and numpy)."""
import ast
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = "paper_2212_02224_gb300"


def _imports(path):
    tree = ast.parse(open(path).read(), filename=path)
    out = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom):
            if node.level == 0 and node.module:
                out.add(node.module.split(".")[0])
    return out


def test_oracle_imports_nothing_from_the_product():
    for path in glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        assert PKG not in _imports(path), path


def test_product_never_imports_the_oracle():
    for path in glob.glob(os.path.join(ROOT, PKG, "*.py")):
        assert "oracle" not in _imports(path), path
    for path in glob.glob(os.path.join(ROOT, PKG, "csrc", "*")) + glob.glob(
            os.path.join(ROOT, "include", "*.h")):
        text = open(path).read()
        assert not re.search(r'#include\s*[<"][^>"]*oracle', text), path


def test_input_generator_module_imports_only_the_standard_library_and_numpy():
    path = os.path.join(ROOT, PKG, "scenegen.py")
    assert _imports(path) <= {"__future__", "dataclasses", "math", "numpy"}, _imports(path)
