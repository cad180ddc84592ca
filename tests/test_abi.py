"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/fsmp.h declares (CPU only: no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "fsmp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fsmp_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for required in ("fsmp_create", "fsmp_submit", "fsmp_poll", "fsmp_destroy", "fsmp_strerror",
                     "fsmp_run_device"):
        assert required in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2403_03156_gb300 import build, fsmp
    path = build.build()
    L = ctypes.CDLL(path)
    for name in declared_entry_points():
        assert hasattr(L, name), name
    assert sorted(fsmp.EXPORTS) == declared_entry_points()


def test_strerror_without_gpu():
    from paper_2403_03156_gb300 import fsmp
    assert fsmp.strerror(fsmp.ERR_BUSY) == "submit queue full"
    assert fsmp.strerror(12345) == "unknown status"


def test_struct_sizes_match_header_layout():
    from paper_2403_03156_gb300 import fsmp
    assert fsmp.SUMMARY_DTYPE.itemsize == 11 * 8 + 14 * 4
    assert fsmp.TRACE_DTYPE.itemsize == 5 * 8 + 4 * 4


def test_binding_refuses_to_run_without_library(monkeypatch, tmp_path):
    from paper_2403_03156_gb300 import fsmp
    monkeypatch.setattr(fsmp, "_lib", None)
    monkeypatch.setattr(fsmp, "lib_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        fsmp.load()
