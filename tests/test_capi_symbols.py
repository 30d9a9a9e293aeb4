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


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every ctypes struct of the binding has the size and field offsets that
    a C compiler gives the header's struct of the same name."""
    import shutil
    import subprocess

    import paper_1702_02939_gb300 as cg

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [cg.cg_replica, cg.cg_params, cg.cg_launch, cg.cg_avm_params, cg.cg_counters]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "cellgb.h"', "int main(void) {"]
    for s in structs:
        name = s.__name__
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in s._fields_:
            lines.append(f'  printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                        text=True).stdout.splitlines())
    for s in structs:
        name = s.__name__
        assert int(got[name]) == ctypes.sizeof(s), name
        for f, _ in s._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(s, f).offset, (name, f)
