"""The GPU path and the oracle are independent: the package neither imports
nor includes anything of oracle/, the oracle nothing of the package, the
shared input generator holds no method arithmetic, and the package has no
CPU fallback -- without its library it fails loudly."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def sources(folder, exts):
    for dp, _, fs in os.walk(os.path.join(ROOT, folder)):
        if "/lib" in dp or "__pycache__" in dp:
            continue
        for f in fs:
            if f.endswith(exts):
                yield os.path.join(dp, f), open(os.path.join(dp, f), errors="replace").read()


def test_package_does_not_use_the_oracle():
    for path, src in sources("paper_1310_0956_gb300", (".py", ".cu", ".cuh", ".h")):
        assert not re.search(r"^\s*(import|from)\s+oracle\b", src, flags=re.M), path
        assert "wmg_oracle" not in src and "liboracle" not in src, path
    for path, src in sources("include", (".h",)):
        assert "oracle" not in src, path


def test_oracle_does_not_use_the_package():
    for path, src in sources("oracle", (".py", ".c", ".h")):
        assert not re.search(r"^\s*(import|from)\s+paper_1310_0956_gb300\b", src, flags=re.M), path
        assert "wmgct.h" not in src and "libwmgct" not in src, path


def test_generator_holds_no_method_arithmetic():
    src = open(os.path.join(ROOT, "synthetic", "__init__.py")).read()
    assert not re.search(r"^\s*(import|from)\s+(oracle|paper_1310_0956_gb300)\b", src, flags=re.M)
    for word in ("project", "backproject", "haar", "cgls", "gmres", "bicgstab"):
        assert not re.search(rf"def\s+\w*{word}\w*\s*\(", src, flags=re.I), word


def test_no_fallback_without_the_library(monkeypatch):
    pytest.importorskip("torch")
    import paper_1310_0956_gb300 as wmg

    def no_toolkit(*a, **k):
        raise RuntimeError("nvcc not found")
    monkeypatch.setattr(wmg, "_lib", None)
    monkeypatch.setattr(wmg._build, "build", no_toolkit)
    with pytest.raises(RuntimeError):
        wmg.lib()
