"""The product path has no CPU fallback: without libptg.so every call raises,
and the package never loads the oracle (which is test infrastructure)."""
import os
import subprocess
import sys

import pytest

import paper_1610_03525_gb300 as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_calls_fail_loudly_without_the_library(monkeypatch, tmp_path):
    monkeypatch.setattr(P, "LIB_PATH", str(tmp_path / "libptg.so"))
    monkeypatch.setattr(P, "_lib", None)
    d = P.make_desc()
    with pytest.raises(RuntimeError, match="not built"):
        P.ptg_validate(d)
    with pytest.raises(RuntimeError, match="not built"):
        P.ptg_create(0)


def test_package_does_not_load_the_oracle():
    code = ("import sys, paper_1610_03525_gb300 as P, paper_1610_03525_gb300.workloads, "
            "paper_1610_03525_gb300.roofline; P.make_desc(); print(sorted(m for m in sys.modules "
            "if m == 'oracle' or m.startswith('oracle.')))")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, check=True)
    assert out.stdout.strip() == "[]"
    pkg = os.path.join(ROOT, "paper_1610_03525_gb300")
    for name in os.listdir(pkg):
        if name.endswith(".py"):
            text = open(os.path.join(pkg, name)).read()
            assert "import oracle" not in text and "from oracle" not in text, name
