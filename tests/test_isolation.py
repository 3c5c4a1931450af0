"""The product path and the oracle stay apart, and the product path has no
CPU fallback.

The CUDA library and its binding never import, include or call the oracle;
the oracle never imports the library; only the seeded input generators
(``synth.py``, no search arithmetic) serve both.  When the CUDA library
cannot be built or loaded, the binding raises instead of computing anything
on the CPU.
"""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2512_00398_gb300")


def _sources(top, exts):
    for d, _, files in os.walk(top):
        if "__pycache__" in d or "_build" in d:
            continue
        for f in files:
            if f.endswith(exts):
                yield os.path.join(d, f)


def _code(path):
    src = open(path).read()
    if path.endswith(".py"):
        src = re.sub(r'""".*?"""', "", src, flags=re.S)   # docstrings may name the oracle
        src = re.sub(r"#.*", "", src)
    else:
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//.*", "", src)
    return src


def test_library_never_references_the_oracle():
    files = list(_sources(PKG, (".py", ".cu", ".cuh", ".cpp", ".h")))
    files += list(_sources(os.path.join(ROOT, "include"), (".h",)))
    assert len(files) > 10
    for f in files:
        code = _code(f)
        assert not re.search(r"\boracle\b|hpo_|hp_oracle", code), f


def test_oracle_never_references_the_library():
    for f in _sources(os.path.join(ROOT, "oracle"), (".py", ".c", ".h")):
        code = _code(f)
        assert not re.search(r"paper_2512_00398_gb300|libhp\b|\bhp_[a-z]+\(|csrc", code), f


def test_no_cpu_fallback_when_the_library_is_missing(monkeypatch):
    import paper_2512_00398_gb300._lib as L

    def no_library(*a, **k):
        raise RuntimeError("nvcc failed")

    monkeypatch.setattr(L, "_lib", None)
    monkeypatch.setattr(L._build, "build", no_library)
    with pytest.raises(RuntimeError):
        L.lib()
    monkeypatch.setattr(L._build, "build", lambda *a, **k: "/nonexistent/libhp.so")
    with pytest.raises(OSError):
        L.lib()
