"""The C-ABI library loads without a GPU and exports every entry point that
include/rbsog.h declares (no compute calls are made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:int|void|const\s+char\s*\*|rbsog_ctx\s*\*)\s*\**\s*(rbsog_\w+)\s*\(",
                                src, flags=re.M)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared()
    for must in ("rbsog_create", "rbsog_set_system", "rbsog_compute_forces", "rbsog_step"):
        assert must in names


def test_library_exports_all_declared():
    from paper_2512_24970_gb300 import build, rbsog
    try:
        build.nvcc()
    except RuntimeError:
        pytest.skip("no CUDA toolkit")
    build.build()
    lib = ctypes.CDLL(build.LIB)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(rbsog.EXPORTS) == declared()


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2512_24970_gb300 import rbsog
    monkeypatch.setattr(rbsog, "_lib", None)
    monkeypatch.setattr(rbsog, "lib_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        rbsog.load()
