"""The product path never routes through the oracle, and fails loudly
without its CUDA library (no CPU fallback)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2606_21784_gb300")


def test_package_never_imports_the_oracle():
    for dirpath, _, files in os.walk(PKG):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, fn)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, re.M), fn
                assert "ks_oracle" not in src and "ko_" not in src, fn


def test_oracle_shares_no_source_with_the_library():
    src = open(os.path.join(ROOT, "oracle", "ks_oracle.c")).read()
    assert "#include \"ks_" not in src and "kineticsim.h" not in src


def test_binding_raises_without_the_library(monkeypatch, tmp_path):
    from paper_2606_21784_gb300 import build as b
    from paper_2606_21784_gb300 import kineticsim as ks
    monkeypatch.setattr(ks, "_lib", None)
    monkeypatch.setattr(b, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        ks.load(build_if_missing=False)
