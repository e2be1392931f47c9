"""The C-ABI library loads and exports every entry point include/dpf.h declares
(CPU only: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "dpf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dpf_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libdpf():
    from paper_1203_2394_gb300 import build
    return ctypes.CDLL(build.build())


def test_every_declared_symbol_is_exported(libdpf):
    names = declared()
    assert "dpf_create" in names and "dpf_resample" in names and "dpf_step" in names
    for n in names:
        assert hasattr(libdpf, n), n


def test_binding_signatures_cover_header():
    from paper_1203_2394_gb300 import dpf
    assert sorted(n for n, _, _ in dpf.SIGNATURES) == declared()


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_1203_2394_gb300 import dpf
    monkeypatch.setattr(dpf, "_lib", None)
    monkeypatch.setattr(dpf, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(dpf.DpfLibraryMissing):
        dpf.lib()
