"""Static check that the oracle and the CUDA path stay apart: the product
package never imports the oracle and its sources never include or load it;
the oracle includes nothing of the product; bench.py touches the oracle only
in the function that times it, and __graft_entry__ only in build() and
smoke()."""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2112_03229_gb300")


def imports_of(tree):
    """(module name, enclosing function or None) for every import in a module."""
    out = []

    def visit(node, fn):
        for child in ast.iter_child_nodes(node):
            name = child.name if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)) else fn
            if isinstance(child, ast.Import):
                out.extend((a.name, fn) for a in child.names)
            elif isinstance(child, ast.ImportFrom) and child.module:
                out.append((child.module, fn))
            visit(child, name)

    visit(tree, None)
    return out


def parse(path):
    with open(path) as f:
        return ast.parse(f.read(), path)


def test_product_package_never_imports_the_oracle():
    for dirpath, _, files in os.walk(PKG):
        for f in files:
            path = os.path.join(dirpath, f)
            if f.endswith(".py"):
                for mod, _ in imports_of(parse(path)):
                    assert mod.split(".")[0] != "oracle", (path, mod)
            elif f.endswith((".cu", ".cuh", ".h")):
                text = open(path).read()
                assert not re.search(r'#include\s*[<"][^>"]*oracle', text), path
                assert "liboracle" not in text, path


def test_oracle_includes_nothing_of_the_product():
    text = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    includes = re.findall(r'#include\s*[<"]([^>"]+)[>"]', text)
    assert includes and all("/" not in i and not i.startswith(("ss_", "simdsearch", "plan")) for i in includes), includes
    for f in ("__init__.py", "build.py"):
        for mod, _ in imports_of(parse(os.path.join(ROOT, "oracle", f))):
            assert mod.split(".")[0] not in ("paper_2112_03229_gb300", "torch"), (f, mod)


def test_bench_and_entry_touch_the_oracle_only_where_allowed():
    bench = [(m, fn) for m, fn in imports_of(parse(os.path.join(ROOT, "bench.py"))) if m.split(".")[0] == "oracle"]
    assert bench and all(fn == "_oracle_call" for _, fn in bench), bench
    entry = [(m, fn) for m, fn in imports_of(parse(os.path.join(ROOT, "__graft_entry__.py")))
             if m.split(".")[0] == "oracle"]
    assert entry and all(fn in ("build", "smoke") for _, fn in entry), entry
