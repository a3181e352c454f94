"""Seeded synthetic hexahedral meshes stored as unstructured lists.

This module only builds connectivity and node coordinates (the inputs of
``fvs_mesh_create``); it holds none of the finite-volume arithmetic, so both
the CUDA path and the CPU oracle can take their inputs from it.

A box mesh has ``nx*ny*nz`` hexahedra.  Its lists follow the conventions of the
finite-volume method of the paper's Section 2.3 (Fig. 1):

* ``nodes``      float64 [Nv, 3]
* ``cells``      int32   [Nc, 8]   hexahedron corners in VTK order
* ``faces``      int32   [Nf, 4]   face corners V1..V4 in cyclic order, oriented
                                   so that the right-hand normal points from the
                                   owner cell C1 to the neighbour C2 (outward on
                                   boundary faces); V1V3 and V2V4 are the face
                                   diagonals used as the local eta/zeta axes
* ``face_cells`` int32   [Nf, 2]   (owner C1, neighbour C2), C2 = -1 on the boundary
* ``patch``      int32   [Nf]      -1 interior; 0..5 = x0, x1, y0, y1, z0, z1 walls

Interior nodes may be jittered (uniform, a fraction of the local spacing per
axis) and cells, faces and nodes may be randomly renumbered, both from seeds.
"""
from __future__ import annotations

import numpy as np

PATCH_X0, PATCH_X1, PATCH_Y0, PATCH_Y1, PATCH_Z0, PATCH_Z1 = range(6)


def box_mesh(nx, ny, nz, lengths=(0.1, 0.1, 0.0125), jitter=0.0, jitter_seed=0,
             permute_seed=None, mirror_z=False, distort=0.0):
    """Build a box of ``nx*ny*nz`` hexahedra.

    ``jitter``: interior nodes move by U(-jitter, jitter) times the cell width
    along each axis (boundary nodes stay put, so the walls remain planar).
    ``permute_seed``: if not None, cells, faces and nodes are renumbered by
    random permutations drawn from this seed.
    ``distort``: smooth non-orthogonal mapping of the whole box; node
    displacements are ``distort`` times the box length along each axis times
    products of sines, vanishing in the normal direction on every wall (so the
    walls stay planar) and refining smoothly with the mesh.
    ``mirror_z``: reflect every node of the (jittered) mesh in the plane
    z = Lz/2 while keeping all ids, so that cell c of the mirrored mesh is the
    reflection of cell c of the original one and a solution on the mirrored
    mesh must equal the reflection of the solution on the original.
    """
    Lx, Ly, Lz = (float(v) for v in lengths)
    hx, hy, hz = Lx / nx, Ly / ny, Lz / nz
    NX, NY, NZ = nx + 1, ny + 1, nz + 1

    def nid(i, j, k):
        return i + NX * (j + NY * k)

    ii, jj, kk = np.meshgrid(np.arange(NX), np.arange(NY), np.arange(NZ), indexing="ij")
    ii = ii.transpose(2, 1, 0).ravel()  # node id order: i fastest, then j, then k
    jj = jj.transpose(2, 1, 0).ravel()
    kk = kk.transpose(2, 1, 0).ravel()
    nodes = np.stack([ii * hx, jj * hy, kk * hz], axis=1).astype(np.float64)

    if distort > 0.0:
        u, v, w = ii / nx, jj / ny, kk / nz
        nodes[:, 0] += distort * Lx * np.sin(np.pi * u) * np.sin(np.pi * v + 0.5) * np.cos(np.pi * w)
        nodes[:, 1] += distort * Ly * np.sin(np.pi * v) * np.sin(np.pi * w + 0.5) * np.cos(np.pi * u)
        nodes[:, 2] += distort * Lz * np.sin(np.pi * w) * np.sin(np.pi * u + 0.5) * np.cos(np.pi * v)
    if jitter > 0.0:
        rng = np.random.default_rng(jitter_seed)
        disp = rng.uniform(-jitter, jitter, size=(NX, NY, NZ, 3))
        interior = (ii > 0) & (ii < nx) & (jj > 0) & (jj < ny) & (kk > 0) & (kk < nz)
        d = disp[ii, jj, kk] * np.array([hx, hy, hz])
        nodes[interior] += d[interior]
    if mirror_z:
        nodes[:, 2] = Lz - nodes[:, 2]

    # cells, VTK hexahedron order
    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ci = ci.transpose(2, 1, 0).ravel()
    cj = cj.transpose(2, 1, 0).ravel()
    ck = ck.transpose(2, 1, 0).ravel()
    cells = np.stack([
        nid(ci, cj, ck), nid(ci + 1, cj, ck), nid(ci + 1, cj + 1, ck), nid(ci, cj + 1, ck),
        nid(ci, cj, ck + 1), nid(ci + 1, cj, ck + 1), nid(ci + 1, cj + 1, ck + 1), nid(ci, cj + 1, ck + 1),
    ], axis=1)

    def cid(i, j, k):
        return i + nx * (j + ny * k)

    faces, fcells, patch = [], [], []

    # x-faces at i = 0..nx; corner order gives a +x normal
    fi, fj, fk = (a.ravel() for a in np.meshgrid(np.arange(NX), np.arange(ny), np.arange(nz), indexing="ij"))
    quad = np.stack([nid(fi, fj, fk), nid(fi, fj + 1, fk), nid(fi, fj + 1, fk + 1), nid(fi, fj, fk + 1)], axis=1)
    own = np.where(fi > 0, cid(fi - 1, fj, fk), cid(0, fj, fk))
    nei = np.where((fi > 0) & (fi < nx), cid(np.minimum(fi, nx - 1), fj, fk), -1)
    pat = np.where(fi == 0, PATCH_X0, np.where(fi == nx, PATCH_X1, -1))
    quad = np.where((fi == 0)[:, None], quad[:, ::-1], quad)  # outward (-x) on the x0 wall
    faces.append(quad); fcells.append(np.stack([own, nei], 1)); patch.append(pat)

    # y-faces at j = 0..ny; +y normal
    fi, fj, fk = (a.ravel() for a in np.meshgrid(np.arange(nx), np.arange(NY), np.arange(nz), indexing="ij"))
    quad = np.stack([nid(fi, fj, fk), nid(fi, fj, fk + 1), nid(fi + 1, fj, fk + 1), nid(fi + 1, fj, fk)], axis=1)
    own = np.where(fj > 0, cid(fi, fj - 1, fk), cid(fi, 0, fk))
    nei = np.where((fj > 0) & (fj < ny), cid(fi, np.minimum(fj, ny - 1), fk), -1)
    pat = np.where(fj == 0, PATCH_Y0, np.where(fj == ny, PATCH_Y1, -1))
    quad = np.where((fj == 0)[:, None], quad[:, ::-1], quad)
    faces.append(quad); fcells.append(np.stack([own, nei], 1)); patch.append(pat)

    # z-faces at k = 0..nz; +z normal
    fi, fj, fk = (a.ravel() for a in np.meshgrid(np.arange(nx), np.arange(ny), np.arange(NZ), indexing="ij"))
    quad = np.stack([nid(fi, fj, fk), nid(fi + 1, fj, fk), nid(fi + 1, fj + 1, fk), nid(fi, fj + 1, fk)], axis=1)
    own = np.where(fk > 0, cid(fi, fj, fk - 1), cid(fi, fj, 0))
    nei = np.where((fk > 0) & (fk < nz), cid(fi, fj, np.minimum(fk, nz - 1)), -1)
    pat = np.where(fk == 0, PATCH_Z0, np.where(fk == nz, PATCH_Z1, -1))
    quad = np.where((fk == 0)[:, None], quad[:, ::-1], quad)
    faces.append(quad); fcells.append(np.stack([own, nei], 1)); patch.append(pat)

    faces = np.concatenate(faces).astype(np.int64)
    face_cells = np.concatenate(fcells).astype(np.int64)
    patch = np.concatenate(patch).astype(np.int64)
    if mirror_z:
        # reflection reverses orientation: flip the corner cycle of every face
        # (V1 stays first, so the eta/zeta diagonals keep their roles) and the
        # corner order of every cell (swap bottom and top quads)
        faces = faces[:, [0, 3, 2, 1]]
        cells = cells[:, [4, 5, 6, 7, 0, 1, 2, 3]]

    cell_ijk = np.stack([ci, cj, ck], axis=1)
    if permute_seed is not None:
        rng = np.random.default_rng(permute_seed)
        pc = rng.permutation(len(cells))      # new cell id -> old cell id
        pf = rng.permutation(len(faces))
        pn = rng.permutation(len(nodes))
        inv_c = np.empty_like(pc); inv_c[pc] = np.arange(len(pc))
        inv_n = np.empty_like(pn); inv_n[pn] = np.arange(len(pn))
        nodes = nodes[pn]
        cells = inv_n[cells[pc]]
        cell_ijk = cell_ijk[pc]
        faces = inv_n[faces[pf]]
        fc = face_cells[pf]
        face_cells = np.where(fc >= 0, inv_c[np.maximum(fc, 0)], -1)
        patch = patch[pf]

    return dict(
        nodes=np.ascontiguousarray(nodes, dtype=np.float64),
        cells=np.ascontiguousarray(cells, dtype=np.int32),
        faces=np.ascontiguousarray(faces, dtype=np.int32),
        face_cells=np.ascontiguousarray(face_cells, dtype=np.int32),
        patch=np.ascontiguousarray(patch, dtype=np.int32),
        cell_ijk=np.ascontiguousarray(cell_ijk, dtype=np.int32),
        shape=(nx, ny, nz),
        lengths=(Lx, Ly, Lz),
    )


def strip_mesh(n, length=0.1, width=1e-3):
    """A 1-D column of ``n`` cells along x (one cell in y and z)."""
    return box_mesh(n, 1, 1, lengths=(length, width, width))


def zones_inner_box(mesh, lo, hi):
    """Cell zones for a metal block inside a mold: 0 (metal) where the cell
    centre lies inside the box [lo, hi], 1 (mold) elsewhere.  int32 [Nc]."""
    X = np.asarray(mesh["nodes"], dtype=np.float64)
    xc = X[np.asarray(mesh["cells"])].mean(axis=1)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    inside = np.all((xc >= lo) & (xc <= hi), axis=1)
    return np.where(inside, 0, 1).astype(np.int32)
