"""fvs_query_fields_noalloc returns what fvs_query_fields returns.

The no-allocation read-back is for callers that cannot allocate GPU memory
(a monitoring thread that must not block in the allocator, or a process
whose device memory is fully committed); it stages the field in a fixed
device array.  Collected last on purpose (file name), so that a failure here
does not hide the results of the other GPU tests.
"""
import ctypes as C

import numpy as np
import pytest

from fvs_inputs import box_mesh, cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fvs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import os
    from paper_1810_08572_gb300 import LIB_PATH, build
    if not os.path.exists(LIB_PATH):
        build()
    from paper_1810_08572_gb300 import fvs as f
    return f


def noalloc(fvs, S, name, n):
    out = np.full(n, np.nan)
    r = fvs.fvs_query_fields_noalloc(S.h, fvs.FIELDS[name], out.ctypes.data_as(C.c_void_p), n)
    assert r == fvs.FVS_OK, fvs.fvs_last_error()
    return out


def test_noalloc_matches_query_fields_on_two_calls(fvs):
    m = box_mesh(12, 10, 3, cases.CAVITY, jitter=0.2, jitter_seed=3, permute_seed=4)
    M = fvs.Mesh(m)
    S = fvs.Solver(M, cases.props(grain=dict(kp=0.13, D_s=3e-9, r0=1e-6)))
    nc, nf = M.n_cells, M.n_faces
    sizes = dict(T=nc, FS=nc, U=3 * nc, USTAR=3 * nc, P=nc, FLUX=nf, QOI=4 * nc, CROSS=2 * nc, TAG=nc,
                 FACE_CASE=nf, GRAIN=nc)
    for call in range(2):           # the shared staging array keeps the last call's values
        S.step(1e-3, 3)
        for name, n in sizes.items():
            a = noalloc(fvs, S, name, n)
            b = S.query(name).ravel()
            np.testing.assert_allclose(a, b, rtol=1e-15, atol=0, equal_nan=True, err_msg=name)


def test_noalloc_rejects_oversized_fields(fvs):
    m = box_mesh(110, 100, 32, cases.CAVITY)      # 352,000 cells: U has 1,056,000 values
    M = fvs.Mesh(m)
    S = fvs.Solver(M, cases.props())
    out = np.empty(3 * M.n_cells)
    r = fvs.fvs_query_fields_noalloc(S.h, fvs.FIELDS["U"], out.ctypes.data_as(C.c_void_p), len(out))
    assert r == fvs.FVS_ERR_ARG
    assert "fvs_query_fields" in fvs.fvs_last_error()
    t = noalloc(fvs, S, "T", M.n_cells)     # a field within the limit still works
    np.testing.assert_array_equal(t, S.query("T"))
