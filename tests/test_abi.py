"""The C-ABI library builds, loads and exports every entry point of include/flic.h (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_1311_0861_gb300 import flic

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "flic.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(flic_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(flic.LIB_PATH):
        from paper_1311_0861_gb300 import build
        build.build()
    return flic.load()


def test_header_declares_the_binding_exports():
    assert declared_functions() == sorted(flic.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_version_string(lib):
    assert b"sm_103a" in lib.flic_version()


def test_struct_layouts_match_header(tmp_path):
    """ctypes structures have the C compiler's size and field offsets."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "flic.h"', "int main(void){"]
    for cname, cls in (("flic_grid_desc", flic.GridDesc), ("flic_diag", flic.Diag)):
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            parts = line.split()
            got[(parts[0], parts[1])] = int(parts[2])
    for cname, cls in (("flic_grid_desc", flic.GridDesc), ("flic_diag", flic.Diag)):
        assert got[(cname, "size")] == ctypes.sizeof(cls)
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)


def test_missing_library_fails_loudly(tmp_path):
    saved = flic._lib
    flic._lib = None
    try:
        with pytest.raises(flic.FlicError):
            flic.load(str(tmp_path / "nope.so"))
    finally:
        flic._lib = saved
