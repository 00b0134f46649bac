"""The C-ABI library builds for sm_103a, loads, and exports every symbol the header
declares (no compute calls: this runs without a GPU)."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def lib():
    from paper_2505_10144_gb300 import build
    build.build()
    from paper_2505_10144_gb300 import _lib
    return _lib.load()


def declared_symbols():
    text = (ROOT / "include" / "vrsplat.h").read_text()
    return sorted(set(re.findall(r"^\s*(?:vrs_status|const char\*)\s+(vrs_\w+)\s*\(", text, re.M)))


def test_header_declares_the_binding_list():
    from paper_2505_10144_gb300 import _lib
    assert declared_symbols() == sorted(_lib.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_binding_structs_match_header_sizes():
    from paper_2505_10144_gb300 import _lib
    assert ctypes.sizeof(_lib.Camera) == 12 * 4 + 4 * 4 + 2 * 4 + 4
    assert ctypes.sizeof(_lib.RenderOpts) == 4 + 12 + 4 + 12 + 4
    assert ctypes.sizeof(_lib.Fovea) == 4 * 4 + 2 * 4


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2505_10144_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", tmp_path / "nope.so")
    with pytest.raises(RuntimeError, match="no CPU or PyTorch fallback"):
        _lib.load()
