"""Host part of the line preconditioner of the energy solve (CPU only).

The chains and their storage layout are built by plain C++
(`paper_1810_08572_gb300/csrc/lines_host.h`), compiled here with g++ through
a small shim.  On permuted grid operators whose couplings are strongest
along z the chains must be the z columns; every index the two kernels form
(entry goff[g] + 32 * position + lane for position < llen) must stay inside
the arrays and visit each cell once; the stored slots must point at the
neighbours in the chain; and the kernels' forward and back substitution,
replayed here on the layout, must solve the tridiagonal system exactly.
"""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as sla

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("no C++ compiler")
    out = tmp_path_factory.mktemp("lines") / "liblines.so"
    src = os.path.join(ROOT, "tests", "line_layout_shim.cpp")
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", src, "-o", str(out)], check=True)
    lib = C.CDLL(str(out))
    P = C.c_void_p
    lib.line_layout.argtypes = [P, P, C.c_int64, C.c_int, C.c_int, P, C.c_int64, C.c_int64, P, P, P, P, P]
    lib.line_layout.restype = C.c_int
    return lib


def layout(lib, col, val, n, w, max_line):
    sizes = np.zeros(4, np.int64)
    ptr = lambda a: a.ctypes.data_as(C.c_void_p)
    rc = lib.line_layout(ptr(col), ptr(val), n, w, max_line, ptr(sizes), 0, 0, None, None, None, None, None)
    assert rc == 1 or sizes[1] == 0
    nlines, ngroups, padded, max_len = (int(v) for v in sizes)
    goff = np.zeros(ngroups + 1, np.int64)
    llen = np.zeros(ngroups * 32, np.int32)
    cell = np.zeros(padded, np.int32)
    sprev = np.zeros(padded, np.int8)
    snext = np.zeros(padded, np.int8)
    rc = lib.line_layout(ptr(col), ptr(val), n, w, max_line, ptr(sizes), ngroups, padded, ptr(goff), ptr(llen),
                         ptr(cell), ptr(sprev), ptr(snext))
    assert rc == 0
    return dict(nlines=nlines, ngroups=ngroups, padded=padded, max_len=max_len, goff=goff, llen=llen, cell=cell,
                sprev=sprev, snext=snext)


def grid_operator(nx, ny, nz, cz, seed, periodic_z=False, mass=1.0):
    """7-slot ELL operator of a grid (slot 0 the cell, then -x, +x, -y, +y,
    -z, +z; a missing neighbour is the cell itself with value 0), couplings
    -1, -1.3 and -cz along x, y, z with +-10 % noise, diagonal the sum of
    their magnitudes plus a mass term, cells randomly renumbered.  Returns
    (col, val, diag, ijk) in the new numbering, slot-major."""
    rng = np.random.default_rng(seed)
    n = nx * ny * nz
    perm = rng.permutation(n)          # grid index -> cell id
    i, j, k = np.unravel_index(np.arange(n), (nx, ny, nz))
    w = 7
    col = np.empty((w, n), np.int32)
    val = np.zeros((w, n))
    ids = perm
    col[0, ids] = ids
    base = {0: 1.0, 1: 1.3, 2: cz}
    for s, (ax, d) in enumerate([(0, -1), (0, 1), (1, -1), (1, 1), (2, -1), (2, 1)], start=1):
        c = [i.copy(), j.copy(), k.copy()]
        c[ax] = c[ax] + d
        dims = (nx, ny, nz)
        if ax == 2 and periodic_z:
            c[2] %= nz
        ok = (c[ax] >= 0) & (c[ax] < dims[ax])
        nbr = np.where(ok, perm[np.ravel_multi_index(tuple(np.clip(c[q], 0, dims[q] - 1) for q in range(3)),
                                                     dims)], ids)
        col[s, ids] = nbr
        val[s, ids] = np.where(ok, -base[ax] * (1.0 + 0.1 * rng.uniform(-1, 1, n)), 0.0)
    # symmetric couplings: average the two directions of each pair
    A = sp.csr_matrix((val.ravel(), (np.tile(np.arange(n), w), col.ravel())), shape=(n, n))
    A.setdiag(0)
    A.eliminate_zeros()
    A = 0.5 * (A + A.T)
    for s in range(1, w):
        val[s] = np.where(val[s] != 0.0, np.asarray(A[np.arange(n), col[s]]).ravel(), 0.0)
    diag = np.abs(val[1:]).sum(0) + mass
    val[0] = diag
    ijk = np.empty((n, 3), np.int64)
    ijk[ids] = np.stack([i, j, k], 1)
    return np.ascontiguousarray(col.ravel()), np.ascontiguousarray(val.ravel()), diag, ijk


def lines_of(L):
    out = []
    for t in range(L["ngroups"] * 32):
        g, lane = divmod(t, 32)
        idx = L["goff"][g] + lane + 32 * np.arange(L["llen"][t], dtype=np.int64)
        assert (idx < L["padded"]).all()
        out.append((t, idx))
    return out


def check_layout(L, col, n, w):
    seen = np.zeros(n, np.int64)
    for t, idx in lines_of(L):
        c = L["cell"][idx]
        assert ((c >= 0) & (c < n)).all()
        seen[c] += 1
        for pos in range(len(idx)):
            sp_, sn_ = int(L["sprev"][idx[pos]]), int(L["snext"][idx[pos]])
            assert (sp_ == -1) == (pos == 0) and (sn_ == -1) == (pos == len(idx) - 1)
            if pos > 0:
                assert 0 <= sp_ < w and col[sp_ * n + c[pos]] == c[pos - 1]
            if pos + 1 < len(idx):
                assert 0 <= sn_ < w and col[sn_ * n + c[pos]] == c[pos + 1]
    assert (seen == 1).all()
    assert (np.diff(L["llen"][: L["nlines"]]) <= 0).all()      # sorted by decreasing length
    assert (L["llen"][L["nlines"]:] == 0).all()


def replay_solve(L, col, val, diag, dextra, r, n):
    """The factor and solve kernels' arithmetic, line by line."""
    z = np.zeros(n)
    for t, idx in lines_of(L):
        c = L["cell"][idx]
        lo = np.array([val[int(L["sprev"][e]) * n + cc] if L["sprev"][e] >= 0 else 0.0 for e, cc in zip(idx, c)])
        up = np.array([val[int(L["snext"][e]) * n + cc] if L["snext"][e] >= 0 else 0.0 for e, cc in zip(idx, c)])
        inv, cp = np.zeros(len(idx)), np.zeros(len(idx))
        cprev = 0.0
        for p in range(len(idx)):
            d = diag[c[p]] + dextra[c[p]] - lo[p] * cprev
            inv[p] = 1.0 / d
            cprev = up[p] * inv[p]
            cp[p] = cprev
        y = 0.0
        for p in range(len(idx)):
            y = (r[c[p]] - lo[p] * y) * inv[p]
            z[c[p]] = y
        x = 0.0
        for p in range(len(idx) - 1, -1, -1):
            x = z[c[p]] - cp[p] * x
            z[c[p]] = x
    return z


def tridiagonal_matrix(L, col, val, diag, dextra, n):
    rows, cols, vals = list(range(n)), list(range(n)), list(diag + dextra)
    for t, idx in lines_of(L):
        c = L["cell"][idx]
        for p, e in enumerate(idx):
            for s, q in ((int(L["sprev"][e]), p - 1), (int(L["snext"][e]), p + 1)):
                if s >= 0:
                    rows.append(c[p])
                    cols.append(c[q])
                    vals.append(val[s * n + c[p]])
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


@pytest.mark.parametrize("max_line", [512, 5])
def test_lines_follow_the_strong_direction(shim, max_line):
    nx, ny, nz = 5, 7, 12
    col, val, diag, ijk = grid_operator(nx, ny, nz, cz=20.0, seed=3)
    n, w = nx * ny * nz, 7
    L = layout(shim, col, val, n, w, max_line)
    check_layout(L, col, n, w)
    expect = [12] * (nx * ny) if max_line >= nz else [5, 5, 2] * (nx * ny)
    assert sorted(L["llen"][: L["nlines"]].tolist()) == sorted(expect)
    for t, idx in lines_of(L):
        c = L["cell"][idx]
        d = np.diff(ijk[c], axis=0)
        assert (d[:, :2] == 0).all() and (np.abs(d[:, 2]) == 1).all()   # one z column, consecutive cells
    rng = np.random.default_rng(4)
    dextra = rng.uniform(0.0, 2.0, n)
    r = rng.normal(size=n)
    z = replay_solve(L, col, val, diag, dextra, r, n)
    P = tridiagonal_matrix(L, col, val, diag, dextra, n)
    np.testing.assert_allclose(P @ z, r, rtol=0, atol=1e-12 * np.abs(r).max())
    np.testing.assert_allclose(z, sla.spsolve(P.tocsc(), r), rtol=1e-12, atol=1e-14)


def test_cycles_are_cut_and_ties_stay_valid(shim):
    # periodic z: every cell has two mutual partners, the chains are rings
    nx, ny, nz = 3, 4, 9
    col, val, diag, ijk = grid_operator(nx, ny, nz, cz=20.0, seed=5, periodic_z=True)
    n = nx * ny * nz
    L = layout(shim, col, val, n, 7, 512)
    check_layout(L, col, n, 7)
    assert sorted(L["llen"][: L["nlines"]].tolist()) == [nz] * (nx * ny)
    # isotropic couplings: chains run in whatever direction wins each row,
    # and the layout is still complete and consistent
    col, val, diag, _ = grid_operator(6, 6, 6, cz=1.15, seed=6)
    L = layout(shim, col, val, 216, 7, 512)
    check_layout(L, col, 216, 7)
    rng = np.random.default_rng(7)
    r = rng.normal(size=216)
    z = replay_solve(L, col, val, diag, np.zeros(216), r, 216)
    P = tridiagonal_matrix(L, col, val, diag, np.zeros(216), 216)
    np.testing.assert_allclose(P @ z, r, rtol=0, atol=1e-12 * np.abs(r).max())


def test_lines_on_the_energy_operator_of_thin_jittered_cells(shim):
    """The oracle's energy operator (rho cp V / dt plus half the conduction
    operator of Eq. 4, 27 couplings a row) on a jittered, permuted 6 x 6 x 48
    strip of the bench mesh's thin cells, stored as a slot-major ELL the way
    the library stores it: the chains are the z columns, and BiCGStab
    preconditioned by the kernels' line substitutions (replayed) needs a
    third or less of the iterations point-Jacobi needs."""
    from fvs_inputs import box_mesh, cases
    from oracle.fv import Oracle
    n_side, nz = 6, 48
    h = 0.1 / 128
    m = box_mesh(n_side, n_side, nz, (n_side * h, n_side * h, nz * 0.0125 / 128), jitter=0.2, jitter_seed=31,
                 permute_seed=32)
    o = Oracle(m, cases.props())
    A = (-0.5 * o.LTk + sp.diags(o.rcp * o.g.V / 1e-3)).tocsr()
    A.sort_indices()
    n = A.shape[0]
    w = int(np.diff(A.indptr).max())
    col = np.repeat(np.arange(n, dtype=np.int32)[None, :], w, 0)
    val = np.zeros((w, n))
    for i in range(n):
        lo, hi = A.indptr[i], A.indptr[i + 1]
        col[: hi - lo, i] = A.indices[lo:hi]
        val[: hi - lo, i] = A.data[lo:hi]
    col, val = np.ascontiguousarray(col.ravel()), np.ascontiguousarray(val.ravel())
    diag = A.diagonal()
    L = layout(shim, col, val, n, w, 512)
    check_layout(L, col, n, w)
    ijk = m["cell_ijk"]
    for t, idx in lines_of(L):
        c = L["cell"][idx]
        d = np.diff(ijk[c], axis=0)
        assert (d[:, :2] == 0).all() and (np.abs(d[:, 2]) == 1).all()
    assert sorted(L["llen"][: L["nlines"]].tolist()) == [nz] * (n_side * n_side)
    rng = np.random.default_rng(33)
    b = A @ (950.0 + rng.normal(size=n))

    def iterations(apply):
        count = [0]
        x, info = sla.bicgstab(A, b, rtol=1e-10, atol=0.0, maxiter=500,
                               M=sla.LinearOperator(A.shape, matvec=apply),
                               callback=lambda xk: count.__setitem__(0, count[0] + 1))
        assert info == 0 and np.linalg.norm(b - A @ x) <= 1e-9 * np.linalg.norm(b)
        return count[0]

    its_j = iterations(lambda v: v / diag)
    its_l = iterations(lambda v: replay_solve(L, col, val, diag, np.zeros(n), v, n))
    assert its_l * 3 <= its_j, (its_l, its_j)
