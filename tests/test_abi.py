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


def test_struct_layouts_match_header(lib):
    import ctypes as C
    # doubles are 8-aligned, so the int32 members pad as in C
    assert C.sizeof(lib.fvs_patch_bc) == 16
    assert C.sizeof(lib.fvs_material) == 14 * 8
    assert C.sizeof(lib.fvs_step_stats) == 2 * 8 + 4 * 4 + 8 + 5 * 4 + 4 + 8
    assert C.sizeof(lib.fvs_mesh_info) == 4 * 8 + 4 * 4 + 8


def test_null_arguments_are_rejected(lib):
    import ctypes as C
    out = C.c_void_p()
    assert lib.fvs_mesh_create(None, 0, None, 0, None, 0, None, None, 1, None, C.byref(out)) == lib.FVS_ERR_ARG
    assert lib.fvs_step(None, 1e-3, 1, None) == lib.FVS_ERR_ARG
    assert lib.fvs_query_fields(None, 0, None, 0, 0) == lib.FVS_ERR_ARG
