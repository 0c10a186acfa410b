"""The C-ABI library loads and exports every function include/wsconv.h declares (no GPU needed)."""
import ctypes
import os
import re

from conftest import ROOT


def _declared():
    src = open(os.path.join(ROOT, "include", "wsconv.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while")))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("conv_plan", "conv_apply", "ls_solve", "conv_destroy", "conv_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2107_03958_gb300 import _native, build
    build.build()
    lib = ctypes.CDLL(build.LIB)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    # the binding's prototype table covers the same set
    assert set(_native.PROTOTYPES) == set(_declared())


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_2107_03958_gb300 import _native, build
    monkeypatch.setattr(build, "LIB", str(tmp_path / "absent.so"))
    monkeypatch.setattr(_native, "_lib", None)
    import pytest
    with pytest.raises(ImportError):
        _native.load()
