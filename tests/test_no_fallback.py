"""The product path has no CPU fallback: the binding raises when libsgpe.so is
missing, and no file of the package imports, includes or runs the oracle."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2009_13507_gb300")


def test_binding_raises_without_the_library(monkeypatch, tmp_path):
    from paper_2009_13507_gb300 import sgpe
    monkeypatch.setattr(sgpe, "_lib", None)
    monkeypatch.setattr(sgpe, "LIB_PATH", str(tmp_path / "libsgpe.so"))
    with pytest.raises(RuntimeError, match="libsgpe.so not found"):
        sgpe.load()


def test_package_sources_never_reach_the_oracle():
    pat = re.compile(r"\boracle\b|sgpe_oracle|orc_[a-z]")
    hits = []
    for d, _, files in os.walk(PKG):
        if "__pycache__" in d:
            continue
        for f in files:
            if not f.endswith((".py", ".cu", ".cuh", ".h", ".c", ".cpp")):
                continue
            path = os.path.join(d, f)
            for i, line in enumerate(open(path, encoding="utf-8"), 1):
                code = line.split("#", 1)[0] if f.endswith(".py") else line.split("//", 1)[0]
                if re.search(r"^\s*(import|from)\b|#include|dlopen|CDLL|subprocess|exec", code) and pat.search(code):
                    hits.append("%s:%d: %s" % (os.path.relpath(path, ROOT), i, line.strip()))
    assert not hits, hits
