"""CPU checks of the C ABI library: it builds, loads, and exports every entry point that
include/*.h declares; the product code never reaches the reference codec."""
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(gbu_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2111_08692_gb300.build import build
    path = build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (gbu_[a-z0-9_]+)", out))
    declared = _declared()
    assert declared, "no declarations found"
    assert declared <= exported, sorted(declared - exported)


def test_library_loads_with_ctypes():
    import paper_2111_08692_gb300 as g
    L = g.lib()
    for name in _declared():
        assert hasattr(L, name)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    import paper_2111_08692_gb300.binding as b
    monkeypatch.setattr(b, "_lib", None)
    monkeypatch.setattr(b._build, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        b.lib()


def test_product_code_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2111_08692_gb300")
    for f in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
            text = open(f).read()
            assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), f
            assert "gbu_oracle" not in text, f
