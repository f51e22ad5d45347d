"""Where the oracle may be used: tests, __graft_entry__.build() (which compiles the
oracle's C) and smoke(), and bench.py's CPU baseline / reference arm.  The product
package and the C ABI never import, link or name it."""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _product_files():
    for top in ("paper_2512_08465_gb300", "include"):
        for d, _, files in os.walk(os.path.join(ROOT, top)):
            if "__pycache__" in d or "_lib" in d:
                continue
            for f in files:
                if f.endswith((".py", ".cu", ".h", ".cpp", ".c")):
                    yield os.path.join(d, f)


def test_product_never_names_the_oracle():
    pat = re.compile(r"\b(import\s+oracle|from\s+oracle|oracle/|oracle\.)")
    for path in _product_files():
        src = open(path, encoding="utf-8").read()
        assert not pat.search(src), path


def _oracle_import_scopes(path):
    tree = ast.parse(open(path, encoding="utf-8").read())
    scopes = []

    def visit(node, scope):
        for child in ast.iter_child_nodes(node):
            s = child.name if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)) else scope
            if isinstance(child, ast.ImportFrom) and (child.module or "").split(".")[0] == "oracle":
                scopes.append(s)
            if isinstance(child, ast.Import) and any(a.name.split(".")[0] == "oracle" for a in child.names):
                scopes.append(s)
            visit(child, s)
    visit(tree, None)
    return scopes


def test_oracle_imported_only_where_allowed():
    assert set(_oracle_import_scopes(os.path.join(ROOT, "bench.py"))) <= {"cpu_baseline", "run_reference"}
    assert set(_oracle_import_scopes(os.path.join(ROOT, "__graft_entry__.py"))) <= {"build", "smoke"}


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without libcs the binding raises; there is no CPU fallback to return results."""
    import pytest
    from paper_2512_08465_gb300 import build as libbuild
    from paper_2512_08465_gb300 import cs
    monkeypatch.setattr(cs, "_LIB", None)
    monkeypatch.setattr(libbuild, "LIB", str(tmp_path / "libcs.so"))
    with pytest.raises(RuntimeError, match="libcs not found"):
        cs.load_library(build_if_missing=False)
