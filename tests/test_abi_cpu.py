"""CPU-side checks of the boundary: the library builds for sm_103a, loads, and
exports every entry point declared in include/pairf12.h (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(pf12_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2008_03237_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared("pairf12.h")
    assert len(names) >= 11
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_abi():
    from paper_2008_03237_gb300 import _lib
    assert set(_declared("pairf12.h")) == set(_lib.SIGNATURES)


def test_missing_library_fails_loudly(tmp_path):
    from paper_2008_03237_gb300 import _lib
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _lib.load(str(tmp_path / "absent.so"))


def test_generator_library_builds():
    from synthetic import device
    assert os.path.exists(device.build())
