"""Marching cubes on the indicator A at level L (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. III-B: the surface is the isosurface A(q) = L, extracted as a triangle
mesh (vertex positions, normals, connectivity) by marching cubes [35].  The
case table comes from ``oracle.mc_table`` (generated from a face rule).

Readings:
* corner bit = 1 iff A >= L, compared in float64;
* a vertex lies on every grid edge (q, q + e_a) whose end bits differ, at
  t = (L - A_q) / (A_{q+e_a} - A_q), position p(q) + t h_a e_a;
* vertex ids are the rank of (linear node index x + nx (y + ny z), axis)
  among crossing edges; triangles are ordered by cell (linear index of the
  lower corner), then by table order;
* the vertex normal is -grad A, by central differences at the nodes
  (one-sided at the grid border), interpolated with t and normalised.
"""

import numpy as np

from . import conventions as cv
from . import mc_table


def classify(A, L):
    """Cube class per cell [nz-1, ny-1, nx-1] (int64), bit b for corner b."""
    inside = np.asarray(A, dtype=np.float64) >= float(L)
    nz, ny, nx = inside.shape
    cls = np.zeros((nz - 1, ny - 1, nx - 1), dtype=np.int64)
    for b in range(8):
        ox, oy, oz = mc_table.corner_pos(b)
        cls |= inside[oz:oz + nz - 1, oy:oy + ny - 1, ox:ox + nx - 1].astype(np.int64) << b
    return cls


def crossing_edges(A, L):
    """Boolean [nz, ny, nx, 3]: edge (q, q + e_a) crosses the level (False at far faces)."""
    inside = np.asarray(A, dtype=np.float64) >= float(L)
    nz, ny, nx = inside.shape
    cr = np.zeros((nz, ny, nx, 3), dtype=bool)
    cr[:, :, :-1, 0] = inside[:, :, :-1] != inside[:, :, 1:]
    cr[:, :-1, :, 1] = inside[:, :-1, :] != inside[:, 1:, :]
    cr[:-1, :, :, 2] = inside[:-1, :, :] != inside[1:, :, :]
    return cr


def gradient(A, grid_n, bbox):
    """grad A at the nodes [nz, ny, nx, 3]: central differences, one-sided at borders."""
    A = np.asarray(A, dtype=np.float64)
    h = cv.voxel_size(grid_n, bbox)
    g = np.zeros(A.shape + (3,))
    for a, ax in ((0, 2), (1, 1), (2, 0)):   # component a differentiates array axis ax
        n = A.shape[ax]
        fwd = [slice(None)] * 3
        bwd = [slice(None)] * 3
        mid = [slice(None)] * 3
        fwd[ax], bwd[ax], mid[ax] = slice(2, n), slice(0, n - 2), slice(1, n - 1)
        out = np.zeros_like(A)
        out[tuple(mid)] = (A[tuple(fwd)] - A[tuple(bwd)]) / (2.0 * h[a])
        lo0, lo1, hi0, hi1 = [[slice(None)] * 3 for _ in range(4)]
        lo0[ax], lo1[ax], hi0[ax], hi1[ax] = 0, 1, n - 1, n - 2
        out[tuple(lo0)] = (A[tuple(lo1)] - A[tuple(lo0)]) / h[a]
        out[tuple(hi0)] = (A[tuple(hi0)] - A[tuple(hi1)]) / h[a]
        g[..., a] = out
    return g


def marching_cubes(A, L, grid_n, bbox):
    """Return dict(vertices [V,3], normals [V,3], tris [T,3], classes, ntri_per_cell)."""
    A = np.asarray(A, dtype=np.float64)
    L = float(L)
    nz, ny, nx = A.shape
    assert (nx, ny, nz) == tuple(int(v) for v in grid_n)
    h = np.array(cv.voxel_size(grid_n, bbox))
    bmin = np.array([float(b) for b in bbox[:3]])

    cr = crossing_edges(A, L)
    flat_cr = cr.reshape(-1)                       # order: node-major, axis-minor
    vid = np.cumsum(flat_cr) - 1
    vid = np.where(flat_cr, vid, -1).reshape(nz, ny, nx, 3)
    e_idx = np.nonzero(flat_cr)[0]
    node = e_idx // 3
    axis = e_idx % 3
    qx = node % nx
    qy = (node // nx) % ny
    qz = node // (nx * ny)
    q0 = np.stack([qx, qy, qz], axis=1)
    q1 = q0.copy()
    q1[np.arange(len(q1)), axis] += 1
    A0 = A[q0[:, 2], q0[:, 1], q0[:, 0]]
    A1 = A[q1[:, 2], q1[:, 1], q1[:, 0]]
    t = (L - A0) / (A1 - A0)
    pos = bmin + (q0 + 0.5) * h
    pos[np.arange(len(pos)), axis] += t * h[axis]

    g = gradient(A, grid_n, bbox)
    g0 = g[q0[:, 2], q0[:, 1], q0[:, 0]]
    g1 = g[q1[:, 2], q1[:, 1], q1[:, 0]]
    gv = -((1.0 - t)[:, None] * g0 + t[:, None] * g1)
    nrm_len = np.linalg.norm(gv, axis=1)
    nrm = np.zeros_like(gv)
    ok = nrm_len > 0
    nrm[ok] = gv[ok] / nrm_len[ok, None]

    cls = classify(A, L)
    ntri_tab, tri_tab = mc_table.table()
    ntri_cell = ntri_tab[cls]
    cells = np.nonzero(ntri_cell.reshape(-1) > 0)[0]       # increasing cell index
    cnx, cny = nx - 1, ny - 1
    cx = cells % cnx
    cy = (cells // cnx) % cny
    cz = cells // (cnx * cny)
    ccls = cls.reshape(-1)[cells]
    cnt = ntri_tab[ccls]
    tris = []
    # order: by cell, then table order
    maxt = tri_tab.shape[1]
    tri_rows = np.full((len(cells), maxt, 3), -1, dtype=np.int64)
    for k in range(maxt):
        has = cnt > k
        for j in range(3):
            e = tri_tab[ccls[has], k, j]
            off = np.array([mc_table.edge_owner_offset(x) for x in range(12)])[e]
            ax = e // 4
            tri_rows[has, k, j] = vid[cz[has] + off[:, 2], cy[has] + off[:, 1],
                                      cx[has] + off[:, 0], ax]
    tris = tri_rows.reshape(-1, 3)
    tris = tris[tris[:, 0] >= 0]
    assert np.all(tris >= 0), "triangle references an edge without a vertex"
    return {
        "vertices": pos,
        "normals": nrm,
        "tris": tris,
        "classes": cls,
        "ntri_per_cell": ntri_cell,
        "edge_vertex_id": vid,
    }
