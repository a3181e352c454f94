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


def voxel_mesh(mask, h, origin=(0.0, 0.0, 0.0), zone=None):
    """Hexahedral mesh of the True voxels of a boolean array ``mask``
    [nx, ny, nz] with cubic voxels of side ``h`` whose corner (0, 0, 0) sits
    at ``origin``.  Faces between two kept voxels are interior; a face
    between a kept voxel and an empty one (or the array's edge) is a wall
    whose patch is the direction of its outward normal (0..5 = -x, +x, -y, +y,
    -z, +z).  ``zone`` (int array like ``mask``) gives each kept cell its
    ``cell_zone``.  Same list conventions as ``box_mesh``."""
    mask = np.asarray(mask, dtype=bool)
    nx, ny, nz = mask.shape
    NX, NY, NZ = nx + 1, ny + 1, nz + 1
    # cells: ids in (i fastest, then j, then k) order of the kept voxels
    flat = mask.transpose(2, 1, 0).ravel()                  # k-major, i fastest
    cell_of = np.full(flat.shape, -1, dtype=np.int64)
    cell_of[flat] = np.arange(int(flat.sum()))
    cell_of = cell_of.reshape(nz, ny, nx).transpose(2, 1, 0)  # [i, j, k] -> cell id or -1
    # nodes: corners of kept voxels
    used = np.zeros((NX, NY, NZ), dtype=bool)
    for di in (0, 1):
        for dj in (0, 1):
            for dk in (0, 1):
                used[di:di + nx, dj:dj + ny, dk:dk + nz] |= mask
    uflat = used.transpose(2, 1, 0).ravel()
    node_of = np.full(uflat.shape, -1, dtype=np.int64)
    node_of[uflat] = np.arange(int(uflat.sum()))
    node_of = node_of.reshape(NZ, NY, NX).transpose(2, 1, 0)
    ni, nj, nk = (a.transpose(2, 1, 0).ravel()[uflat] for a in
                  np.meshgrid(np.arange(NX), np.arange(NY), np.arange(NZ), indexing="ij"))
    o = np.asarray(origin, dtype=np.float64)
    nodes = np.stack([o[0] + ni * h, o[1] + nj * h, o[2] + nk * h], axis=1)

    ci, cj, ck = np.nonzero(mask.transpose(2, 1, 0))         # k, j, i order ...
    ci, ck = ck, ci                                           # ... back to i, j, k
    cells = np.stack([node_of[ci, cj, ck], node_of[ci + 1, cj, ck], node_of[ci + 1, cj + 1, ck],
                      node_of[ci, cj + 1, ck], node_of[ci, cj, ck + 1], node_of[ci + 1, cj, ck + 1],
                      node_of[ci + 1, cj + 1, ck + 1], node_of[ci, cj + 1, ck + 1]], axis=1)

    pad = np.pad(cell_of, 1, constant_values=-1)              # pad[i+1, j+1, k+1] = cell_of[i, j, k]
    faces, fcells, patch = [], [], []
    for axis in range(3):
        # face positions: index p along the axis (0..n), the others span the voxels
        shape = [nx, ny, nz]
        shape[axis] += 1
        grids = np.meshgrid(*[np.arange(s) for s in shape], indexing="ij")
        lo = [g + 1 for g in grids]
        lo[axis] = grids[axis]                                # voxel below the face (pad coords)
        hi = [g + 1 for g in grids]                           # voxel above the face
        a = pad[lo[0], lo[1], lo[2]].ravel()
        b = pad[hi[0], hi[1], hi[2]].ravel()
        keep = (a >= 0) | (b >= 0)
        fi, fj, fk = (g.ravel()[keep] for g in grids)
        a, b = a[keep], b[keep]
        if axis == 0:
            quad = np.stack([node_of[fi, fj, fk], node_of[fi, fj + 1, fk], node_of[fi, fj + 1, fk + 1],
                             node_of[fi, fj, fk + 1]], axis=1)
        elif axis == 1:
            quad = np.stack([node_of[fi, fj, fk], node_of[fi, fj, fk + 1], node_of[fi + 1, fj, fk + 1],
                             node_of[fi + 1, fj, fk]], axis=1)
        else:
            quad = np.stack([node_of[fi, fj, fk], node_of[fi + 1, fj, fk], node_of[fi + 1, fj + 1, fk],
                             node_of[fi, fj + 1, fk]], axis=1)
        # owner below (normal along +axis); a face with only the voxel above
        # is a wall owned by that voxel, with the corner cycle reversed
        only_hi = a < 0
        own = np.where(only_hi, b, a)
        nei = np.where((a >= 0) & (b >= 0), b, -1)
        quad = np.where(only_hi[:, None], quad[:, ::-1], quad)
        pat = np.where(nei >= 0, -1, np.where(only_hi, 2 * axis, 2 * axis + 1))
        faces.append(quad); fcells.append(np.stack([own, nei], 1)); patch.append(pat)

    out = dict(
        nodes=np.ascontiguousarray(nodes, dtype=np.float64),
        cells=np.ascontiguousarray(cells, dtype=np.int32),
        faces=np.ascontiguousarray(np.concatenate(faces), dtype=np.int32),
        face_cells=np.ascontiguousarray(np.concatenate(fcells), dtype=np.int32),
        patch=np.ascontiguousarray(np.concatenate(patch), dtype=np.int32),
        cell_ijk=np.ascontiguousarray(np.stack([ci, cj, ck], axis=1), dtype=np.int32),
        shape=(nx, ny, nz),
        lengths=(nx * h, ny * h, nz * h),
    )
    if zone is not None:
        out["cell_zone"] = np.ascontiguousarray(np.asarray(zone)[ci, cj, ck], dtype=np.int32)
    return out


def _dilate(mask, s):
    """Grow a boolean voxel set by s voxels along every axis (cube element)."""
    out = mask.copy()
    for axis in range(3):
        src = out.copy()
        for d in range(1, s + 1):
            sl_a = [slice(None)] * 3
            sl_b = [slice(None)] * 3
            sl_a[axis] = slice(d, None)
            sl_b[axis] = slice(None, -d)
            out[tuple(sl_a)] |= src[tuple(sl_b)]
            out[tuple(sl_b)] |= src[tuple(sl_a)]
    return out


def casting_mesh(h, shell=0.003, plate=(0.2, 0.1, 0.02), rib_width=0.005, rib_height=0.01,
                 rib_x=(0.05, 0.10, 0.15), riser=0.02, riser_x=0.18):
    """Voxelised casting in a mold shell: a plate [0, Lx] x [0, Ly] x [0, Lz],
    three ribs of width ``rib_width`` (along x) hanging ``rib_height`` below
    it across the full y span at ``rib_x``, and a cubic riser of side
    ``riser`` on its top face centred at (``riser_x``, Ly/2); all of it metal
    (zone 0) inside a mold shell (zone 1) of every voxel within ``shell`` of
    the metal (cube neighbourhood).  Voxel side ``h``; a voxel is metal when
    its centre lies inside the metal.  The walls of the mesh are the outer
    surface of the shell."""
    Lx, Ly, Lz = plate
    s = max(1, int(round(shell / h)))
    x0, y0, z0 = -shell, -shell, -rib_height - shell
    x1, y1, z1 = Lx + shell, Ly + shell, Lz + riser + shell
    nx, ny, nz = (int(np.ceil((b - a) / h - 1e-9)) for a, b in ((x0, x1), (y0, y1), (z0, z1)))
    xc = x0 + (np.arange(nx) + 0.5) * h
    yc = y0 + (np.arange(ny) + 0.5) * h
    zc = z0 + (np.arange(nz) + 0.5) * h
    X, Y, Z = np.meshgrid(xc, yc, zc, indexing="ij")
    metal = (X > 0) & (X < Lx) & (Y > 0) & (Y < Ly) & (Z > 0) & (Z < Lz)
    for rx in rib_x:
        metal |= (np.abs(X - rx) < 0.5 * rib_width) & (Y > 0) & (Y < Ly) & (Z > -rib_height) & (Z <= 0)
    metal |= ((np.abs(X - riser_x) < 0.5 * riser) & (np.abs(Y - 0.5 * Ly) < 0.5 * riser)
              & (Z >= Lz) & (Z < Lz + riser))
    solid = _dilate(metal, s)
    zone = np.where(metal, 0, 1)
    return voxel_mesh(solid, h, origin=(x0, y0, z0), zone=zone)
