"""The product path's boundary on the CPU: the binding refuses to run without
the CUDA library (no fallback), and no product module imports, loads or runs
the oracle (the oracle is test infrastructure)."""
import ast
import os

import pytest

from paper_2408_12479_gb300 import hx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2408_12479_gb300")


def test_binding_raises_without_the_library(monkeypatch, tmp_path):
    monkeypatch.setattr(hx, "LIB_PATH", str(tmp_path / "missing" / "libhx.so"))
    monkeypatch.setattr(hx, "_lib", None)
    with pytest.raises(ImportError, match="not built"):
        hx.lib()
    with pytest.raises(ImportError):
        hx.hx_fibre_dispersion(3.62, 34.3)


def _product_sources():
    for d, _, files in os.walk(PKG):
        if "_lib" in d.split(os.sep):
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                yield os.path.join(d, f)
    for f in os.listdir(os.path.join(ROOT, "include")):
        yield os.path.join(ROOT, "include", f)


def test_product_never_imports_the_oracle():
    seen = 0
    for path in _product_sources():
        src = open(path, encoding="utf-8").read()
        seen += 1
        if path.endswith(".py"):
            for node in ast.walk(ast.parse(src)):
                if isinstance(node, ast.Import):
                    names = [a.name for a in node.names]
                elif isinstance(node, ast.ImportFrom):
                    names = [node.module or ""]
                else:
                    continue
                assert not any(n == "oracle" or n.startswith("oracle.") for n in names), (path, names)
        # no path into the oracle's sources or its built library
        assert "hx_oracle" not in src and "libhx_oracle" not in src, path
    assert seen >= 10


def test_oracle_shares_nothing_with_the_product():
    """The oracle's Python side imports nothing from the package but (at
    most) the seeded input recipes, and its C source includes only system
    headers."""
    odir = os.path.join(ROOT, "oracle")
    for f in os.listdir(odir):
        path = os.path.join(odir, f)
        if f.endswith(".py"):
            for node in ast.walk(ast.parse(open(path, encoding="utf-8").read())):
                mods = []
                if isinstance(node, ast.Import):
                    mods = [a.name for a in node.names]
                elif isinstance(node, ast.ImportFrom):
                    mods = [(node.module or "") + "." + a.name for a in node.names]
                for mname in mods:
                    if mname.startswith("paper_2408_12479_gb300"):
                        assert mname == "paper_2408_12479_gb300.inputs", (f, mname)
        elif f.endswith((".c", ".h")):
            for line in open(path, encoding="utf-8"):
                if line.lstrip().startswith("#include"):
                    assert "<" in line and '"' not in line, (f, line)
