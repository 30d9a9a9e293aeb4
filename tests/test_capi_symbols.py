"""The C-ABI library builds, loads without a GPU and exports every entry point
declared in include/*.h (no compute call is made here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(cg_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("cg_create", "cg_step", "cg_get_state", "cg_get_neighbors", "cg_set_p0", "cg_set_v0",
                 "cg_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol():
    import paper_1702_02939_gb300 as cg
    from paper_1702_02939_gb300 import _build

    _build.build()
    L = ctypes.CDLL(_build.LIB)
    missing = [n for n in sorted(declared_functions()) if not hasattr(L, n)]
    assert not missing, missing
    assert cg.lib() is not None


def test_status_strings_without_gpu():
    import paper_1702_02939_gb300 as cg

    L = cg.lib()
    for code in range(-9, 1):
        assert L.cg_status_string(code)


def test_workspace_size_is_host_only():
    import paper_1702_02939_gb300 as cg

    b1 = cg.cg_workspace_bytes([dict(n=400, Lx=20, Ly=20, p0=3.8, v0=0.05)])
    b2 = cg.cg_workspace_bytes([dict(n=800, Lx=20, Ly=40, p0=3.8, v0=0.05)])
    assert 0 < b1 < b2
    with pytest.raises(cg.CellgbError):
        cg.cg_workspace_bytes([dict(n=4, Lx=2, Ly=2, p0=3.8, v0=0.05)])
