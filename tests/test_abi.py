"""The C-ABI library builds, loads without a GPU and exports every declared entry point."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    with open(os.path.join(ROOT, "include", "dclno.h")) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dclno_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_declared_symbols():
    from paper_1809_05637_gb300 import build as b
    b.build()
    import paper_1809_05637_gb300 as pkg
    decl = declared_symbols()
    assert decl, "no declarations found"
    assert set(decl) == set(pkg._lib.SYMBOLS), "binding symbol list out of date"
    lib = pkg.load_library()
    for name in decl:
        assert hasattr(lib, name), name


def test_no_cpu_fallback_without_library(tmp_path, monkeypatch):
    import paper_1809_05637_gb300._lib as L
    monkeypatch.setattr(L, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(L, "_LIB", None)
    with pytest.raises(ImportError):
        L.load_library()
