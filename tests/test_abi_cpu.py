"""The C-ABI library builds for sm_103a, loads, and exports every symbol the header
declares (no compute calls: this runs without a GPU)."""
import ctypes
import re
import subprocess
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


def test_binding_structs_match_header_sizes(tmp_path):
    """Sizes and field offsets of the ctypes mirrors equal what a C compiler lays out for
    the header's structs."""
    from paper_2505_10144_gb300 import _lib
    pairs = {"vrs_gaussians": _lib.Gaussians, "vrs_gaussian_grads": _lib.GaussianGrads,
             "vrs_camera": _lib.Camera, "vrs_fovea": _lib.Fovea, "vrs_render_opts": _lib.RenderOpts, "vrs_peaks": _lib.Peaks}
    lines = ['#include <stdio.h>', '#include "vrsplat.h"', "int main(void) {"]
    for cname, cls in pairs.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for f in cls._fields_:
            lines.append(f'  printf("{cname}.{f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "abi.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "abi"
    subprocess.run(["gcc", "-std=c11", "-I", str(ROOT / "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    for cname, cls in pairs.items():
        assert int(got[cname]) == ctypes.sizeof(cls), cname
        for f in cls._fields_:
            assert int(got[f"{cname}.{f[0]}"]) == getattr(cls, f[0]).offset, (cname, f[0])


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2505_10144_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", tmp_path / "nope.so")
    with pytest.raises(RuntimeError, match="no CPU or PyTorch fallback"):
        _lib.load()
