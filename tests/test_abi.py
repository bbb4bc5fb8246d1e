"""The C-ABI library builds, loads and exports every function include/*.h declares (no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s+\**([a-z][a-z0-9_]*)\s*\(", txt, re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2109_12390_gb300.build import build
    path = build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = _declared()
    for required in ("mpm_init", "mpm_step", "mpm_set_state", "mpm_get_state", "mpm_destroy", "mpm_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_python_binding_covers_header(lib):
    from paper_2109_12390_gb300 import _abi
    bound = {s[0] for s in _abi.SIGNATURES}
    assert set(_declared()) <= bound


def test_last_error_is_empty_string_initially(lib):
    lib.mpm_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.mpm_last_error(), bytes)
