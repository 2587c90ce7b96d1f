"""The oracle and the CUDA path share no code, and the product has no CPU
fallback: the oracle imports nothing of the package, the package (Python,
CUDA and C++ sources) imports nothing of the oracle, the seeded inputs
import neither, and the binding refuses to run without its library."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = "paper_1301_0191_gb300"


def _files(top, exts):
    for d, _, names in os.walk(os.path.join(ROOT, top)):
        if "__pycache__" in d or "_build" in d or "_lib" in d:
            continue
        for n in names:
            if n.endswith(exts):
                yield os.path.join(d, n)


def _imports(path):
    src = open(path, encoding="utf-8").read()
    mods = re.findall(r"^\s*(?:from\s+([\w.]+)\s+import|import\s+([\w.]+))", src, flags=re.M)
    return {a or b for a, b in mods}


def test_oracle_imports_nothing_of_the_package():
    for f in _files("oracle", (".py",)):
        bad = {m for m in _imports(f) if m.split(".")[0] in (PKG, "amb_inputs", "torch", "__graft_entry__")}
        assert not bad, (f, bad)


def test_package_imports_nothing_of_the_oracle():
    for f in _files(PKG, (".py",)):
        bad = {m for m in _imports(f) if m.split(".")[0] in ("oracle", "tests", "_work")}
        assert not bad, (f, bad)
    for f in _files(PKG, (".cu", ".cuh", ".h", ".cpp")):
        src = open(f, encoding="utf-8").read()
        assert not re.search(r'#\s*include\s*[<"][^>"]*oracle', src), f


def test_inputs_import_neither_side():
    for f in _files("amb_inputs", (".py",)):
        bad = {m for m in _imports(f) if m.split(".")[0] in (PKG, "oracle")}
        assert not bad, (f, bad)


def test_binding_fails_loudly_without_its_library(monkeypatch):
    from paper_1301_0191_gb300 import binding as B
    monkeypatch.setattr(B, "_lib", None)
    monkeypatch.setattr(B, "LIB", os.path.join(ROOT, "no_such_dir", "libamb.so"))
    with pytest.raises(RuntimeError, match="not built"):
        B.lib()
