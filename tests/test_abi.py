"""The C-ABI library builds, loads, and exports every entry point that
include/fvs.h declares (CPU only: no compute calls)."""
import os
import re

import pytest


@pytest.fixture(scope="module")
def lib(root):
    from paper_1810_08572_gb300 import LIB_PATH, build
    if not os.path.exists(LIB_PATH):
        build()
    from paper_1810_08572_gb300 import fvs
    return fvs


def declared(root):
    text = open(os.path.join(root, "include", "fvs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fvs_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib, root):
    names = declared(root)
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib._lib, n), n
    assert sorted(names) == sorted(lib.EXPORTED)


def test_version_and_error_without_device(lib):
    assert lib.fvs_version().startswith(b"fvs")
    assert isinstance(lib.fvs_last_error(), str)


def test_struct_layouts_match_header(lib, root, tmp_path):
    """Size and every member offset of the binding's ctypes structs equal
    what a C compiler lays out from include/fvs.h."""
    import ctypes as C
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = ["fvs_material", "fvs_patch_bc", "fvs_props", "fvs_step_stats", "fvs_mesh_info", "fvs_uq_options"]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "fvs.h"', "int main(void) {"]
    for name in structs:
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in getattr(lib, name)._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(root, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        a, b, v = line.split()
        got[(a, b)] = int(v)
    for name in structs:
        T = getattr(lib, name)
        assert got[(name, "size")] == C.sizeof(T), name
        for field, _ in T._fields_:
            assert got[(name, field)] == getattr(T, field).offset, (name, field)


def test_null_arguments_are_rejected(lib):
    import ctypes as C
    out = C.c_void_p()
    assert lib.fvs_mesh_create(None, 0, None, 0, None, 0, None, None, 1, None, C.byref(out)) == lib.FVS_ERR_ARG
    assert lib.fvs_step(None, 1e-3, 1, None) == lib.FVS_ERR_ARG
    assert lib.fvs_query_fields(None, 0, None, 0, 0) == lib.FVS_ERR_ARG
