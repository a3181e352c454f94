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


def test_every_entry_point_checks_its_arguments_before_the_device(lib):
    """Each entry point refuses missing handles and impossible sizes with
    FVS_ERR_ARG (or -1 for the counting calls) and a message naming itself,
    before any CUDA call (so this runs without a GPU)."""
    import ctypes as C
    h = C.c_void_p()
    d = C.c_double()
    i32, i64 = C.c_int32(), C.c_int64()
    buf = (C.c_double * 8)()
    ibuf = (C.c_int32 * 8)()
    ARG = lib.FVS_ERR_ARG
    calls = [
        ("fvs_mesh_get_info", (None, None)),
        ("fvs_mesh_geometry", (None, 0, buf, 8)),
        ("fvs_solver_create", (None, None, C.byref(h))),
        ("fvs_set_properties", (None, None)),
        ("fvs_mesh_set_zones", (None, ibuf)),
        ("fvs_set_mold", (None, 7800.0, 500.0, 30.0, 2000.0, 500.0)),
        ("fvs_set_grain_growth", (None, 0.13, 3e-9, 1e-6)),
        ("fvs_set_state", (None, buf, None, 0)),
        ("fvs_step", (None, 1e-3, 1, None)),
        ("fvs_pressure_solve", (None, buf, buf, 1e-8, C.byref(i32), C.byref(d))),
        ("fvs_query_fields", (None, 0, buf, 8, 0)),
        ("fvs_query_fields_noalloc", (None, 0, buf, 8)),
        ("fvs_get_time", (None, C.byref(d), C.byref(i64))),
        ("fvs_profile_enable", (None, 1)),
        ("fvs_profile_read", (None, None, 0, C.byref(i32))),
        ("fvs_uq_batch", (None, None, 4, buf, 1e-3, 10, None, buf, None)),
        ("fvs_surrogate_create", (3, 129, 4, 4, 0, None, C.byref(h))),
        ("fvs_surrogate_create", (3, 128, 0, 4, 0, None, C.byref(h))),
        ("fvs_surrogate_set_scaling", (None, buf, buf, buf, buf)),
        ("fvs_surrogate_params", (None, buf, 8, 0)),
        ("fvs_surrogate_gradients", (None, buf, buf, 1, buf, 8, C.byref(d))),
        ("fvs_surrogate_train", (None, buf, buf, 1, 10, 1e-3, C.byref(d))),
        ("fvs_surrogate_predict", (None, buf, buf, 1, 0)),
        ("fvs_measure_fp64_fma", (0, C.byref(d))),
        ("fvs_pce_create", (0, ibuf, buf, buf, 2, 1, None, C.byref(h))),
        ("fvs_pce_multi_indices", (None, ibuf, 8)),
        ("fvs_pce_nodes", (None, 3, 0, buf, 8, C.byref(i64))),
        ("fvs_pce_fit", (None, buf, buf, 8, C.byref(d))),
        ("fvs_pce_eval", (None, buf, buf, 1, 0)),
        ("fvs_pce_coefficients", (None, buf, 8)),
        ("fvs_pce_sensitivity", (None, buf, buf, buf, buf)),
    ]
    for name, args in calls:
        assert getattr(lib, name)(*args) == ARG, name
        assert lib.fvs_last_error().startswith(name), (name, lib.fvs_last_error())
    for name in ("fvs_mesh_destroy", "fvs_solver_destroy", "fvs_surrogate_destroy", "fvs_pce_destroy"):
        assert getattr(lib, name)(None) == ARG, name
    assert lib.fvs_surrogate_num_params(None) == -1
    assert lib.fvs_pce_num_terms(None) == -1
    # a uniform input (FVS_PCE_UNIFORM = 1 in the header) needs lo < hi
    fam = (C.c_int32 * 1)(1)
    lo, hi = (C.c_double * 1)(1.0), (C.c_double * 1)(1.0)
    assert lib.fvs_pce_create(1, fam, lo, hi, 2, 1, None, C.byref(h)) == ARG
    # ids are 32-bit: a mesh beyond their range is refused before any copy
    nodes = (C.c_double * 3)()
    assert lib.fvs_mesh_create(nodes, 1, ibuf, 200_000_000, ibuf, 1, ibuf, ibuf, 1, None, C.byref(h)) == ARG
    assert "32-bit" in lib.fvs_last_error()
