"""Pins for the oracle marching cubes and its generated table (Sec. III-B, [35]), no GPU."""

import numpy as np
import pytest

from oracle import conventions as cv
from oracle import mc, mc_table as T


def _ambiguous(case):
    bit = [(case >> b) & 1 for b in range(8)]
    for (_, _, cyc, _) in T.faces():
        b = [bit[c] for c in cyc]
        if b[0] == b[2] and b[1] == b[3] and b[0] != b[1]:
            return True
    return False


def test_table_self_consistency():
    ntri, tri = T.table()
    assert ntri[0] == 0 and ntri[255] == 0
    for case in range(256):
        bit = [(case >> b) & 1 for b in range(8)]
        crossed = {e for e in range(12)
                   if bit[T.edge_corners(e)[0]] != bit[T.edge_corners(e)[1]]}
        loops = T.case_loops(case)
        used = [e for lp in loops for e in lp]
        assert sorted(used) == sorted(crossed)          # every crossed edge once
        assert all(len(lp) >= 3 for lp in loops)
        assert ntri[case] == sum(len(lp) - 2 for lp in loops)
        for lp in loops:
            assert lp[0] == min(lp)
        # each directed loop edge (a -> b) lies on a common face of a and b
        for lp in loops:
            for a, b in zip(lp, lp[1:] + lp[:1]):
                fa = {(ax, s) for (ax, s, _, ed) in T.faces() if a in ed}
                fb = {(ax, s) for (ax, s, _, ed) in T.faces() if b in ed}
                assert fa & fb


def test_complement_symmetry_where_unambiguous():
    for case in range(256):
        if _ambiguous(case):
            continue
        a = {frozenset(zip(lp, lp[1:] + lp[:1])) for lp in T.case_loops(case)}
        b = {frozenset((y, x) for (x, y) in zip(lp, lp[1:] + lp[:1]))
             for lp in T.case_loops(255 - case)}
        assert a == b


def _cube_positions(case):
    """Vertex positions at edge midpoints and the triangle normals of one case."""
    pos = {e: np.array(T.edge_mid2(e)) / 2.0 for e in range(12)}
    out = []
    for (a, b, c) in T.case_triangles(case):
        n = np.cross(pos[b] - pos[a], pos[c] - pos[a])
        out.append((a, b, c, n))
    return out


def test_single_cube_orientation():
    """Each loop's vector area points from its inside edge ends to its outside ones."""
    pos = {e: np.array(T.edge_mid2(e)) / 2.0 for e in range(12)}
    for case in range(1, 255):
        bit = [(case >> b) & 1 for b in range(8)]
        tris = T.case_triangles(case)
        k = 0
        for lp in T.case_loops(case):
            area = np.zeros(3)
            for (a, b, c) in tris[k:k + len(lp) - 2]:
                assert {a, b, c} <= set(lp)
                area += np.cross(pos[b] - pos[a], pos[c] - pos[a])
            k += len(lp) - 2
            ins, outs = [], []
            for e in lp:
                c0, c1 = T.edge_corners(e)
                (ins if bit[c0] else outs).append(T.corner_pos(c0))
                (ins if bit[c1] else outs).append(T.corner_pos(c1))
            d = np.mean(outs, axis=0) - np.mean(ins, axis=0)
            assert np.dot(area, d) > 0


def _grid_nodes(grid_n, bbox):
    h = cv.voxel_size(grid_n, bbox)
    nx, ny, nz = grid_n
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return np.stack([bbox[0] + (x + 0.5) * h[0], bbox[1] + (y + 0.5) * h[1],
                     bbox[2] + (z + 0.5) * h[2]], axis=-1)


def test_plane_field_vertices_on_plane():
    grid = (9, 7, 8)
    bbox = (-1, -1, -1, 1, 1, 1)
    P = _grid_nodes(grid, bbox)
    nvec = np.array([0.3, -0.8, 0.5])
    nvec /= np.linalg.norm(nvec)
    A = -(P @ nvec) + 0.05                  # inside where n.p < 0.05; outward normal = n
    m = mc.marching_cubes(A, 0.0, grid, bbox)
    assert len(m["vertices"]) > 0
    assert np.max(np.abs(m["vertices"] @ nvec - 0.05)) < 1e-12
    assert np.allclose(m["normals"], nvec[None, :], atol=1e-12)
    tri = m["tris"]
    v = m["vertices"]
    fn = np.cross(v[tri[:, 1]] - v[tri[:, 0]], v[tri[:, 2]] - v[tri[:, 0]])
    assert np.all(fn @ nvec >= -1e-15)


def test_radial_field_lerp_roots():
    grid = (10, 10, 10)
    bbox = (-1, -1, -1, 1, 1, 1)
    P = _grid_nodes(grid, bbox)
    A = 0.6 - np.linalg.norm(P, axis=-1)
    m = mc.marching_cubes(A, 0.0, grid, bbox)
    # recompute each vertex from the definition: root of the linear interpolant
    vid = m["edge_vertex_id"]
    h = cv.voxel_size(grid, bbox)
    for (z, y, x, a) in zip(*np.nonzero(vid >= 0)):
        q1 = [x, y, z]
        q1[a] += 1
        A0 = A[z, y, x]
        A1 = A[q1[2], q1[1], q1[0]]
        t = A0 / (A0 - A1)
        p = P[z, y, x].copy()
        p[a] += t * h[a]
        assert np.allclose(m["vertices"][vid[z, y, x, a]], p, atol=1e-14)


def _edge_check(tris):
    """(watertight, consistently oriented, Euler characteristic, components)."""
    directed = {}
    for t in tris:
        for a, b in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0])):
            directed[(a, b)] = directed.get((a, b), 0) + 1
    und = {}
    for (a, b), c in directed.items():
        k = (min(a, b), max(a, b))
        und[k] = und.get(k, 0) + c
    watertight = all(c == 2 for c in und.values())
    oriented = all(c == 1 for c in directed.values())
    nv = len(np.unique(tris))
    chi = nv - len(und) + len(tris)
    # components by union-find over triangle vertices
    parent = {v: v for v in np.unique(tris).tolist()}

    def find(v):
        while parent[v] != v:
            parent[v] = parent[parent[v]]
            v = parent[v]
        return v
    for t in tris.tolist():
        for a, b in ((t[0], t[1]), (t[1], t[2])):
            ra, rb = find(a), find(b)
            if ra != rb:
                parent[ra] = rb
    comps = len({find(v) for v in parent})
    return watertight, oriented, chi, comps


@pytest.mark.parametrize("center", [(0.0, 0.0, 0.0), (0.031, -0.017, 0.052)])
def test_analytic_sphere_mesh_is_closed_genus0(center):
    grid = (24, 24, 24)
    bbox = (-1, -1, -1, 1, 1, 1)
    P = _grid_nodes(grid, bbox) - np.array(center)
    A = 0.55 - np.linalg.norm(P, axis=-1)
    m = mc.marching_cubes(A, 0.0, grid, bbox)
    w, o, chi, comps = _edge_check(m["tris"])
    assert w and o and chi == 2 and comps == 1
    v = m["vertices"] - np.array(center)
    assert np.max(np.abs(np.linalg.norm(v, axis=1) - 0.55)) < 2.0 / 24
    tri = m["tris"]
    fn = np.cross(v[tri[:, 1]] - v[tri[:, 0]], v[tri[:, 2]] - v[tri[:, 0]])
    cen = v[tri].mean(axis=1)
    assert np.all(np.einsum("ij,ij->i", fn, cen) > 0)      # outward
    assert np.all(np.einsum("ij,ij->i", m["normals"], v) > 0)


def test_random_fields_are_watertight():
    """Crack-free on random fields: every mesh edge shared by exactly two triangles."""
    rng = np.random.default_rng(4)
    grid = (9, 8, 7)
    bbox = (0, 0, 0, 1, 1, 1)
    for _ in range(5):
        A = rng.standard_normal(grid[::-1])
        A[0, :, :] = A[-1, :, :] = A[:, 0, :] = A[:, -1, :] = A[:, :, 0] = A[:, :, -1] = -5.0
        m = mc.marching_cubes(A, 0.0, grid, bbox)
        w, o, _, _ = _edge_check(m["tris"])
        assert w and o


def test_all_single_cube_cases_close_with_padding():
    """Each of the 256 cases in a padded 4^3 field yields a closed oriented mesh."""
    for case in range(1, 255):
        A = -np.ones((4, 4, 4))
        for b in range(8):
            ox, oy, oz = T.corner_pos(b)
            A[1 + oz, 1 + oy, 1 + ox] = 1.0 if (case >> b) & 1 else -1.0
        m = mc.marching_cubes(A, 0.0, (4, 4, 4), (0, 0, 0, 1, 1, 1))
        assert m["classes"][1, 1, 1] == case
        w, o, _, _ = _edge_check(m["tris"])
        assert w and o
