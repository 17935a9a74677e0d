"""Marching-cubes case table generated from a face rule (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. III-B extracts the surface A = L "using the marching cubes algorithm
[35]" and prints no table.  The table is therefore generated here from a
stated rule rather than copied:

Cube numbering.  Corner b in 0..7 sits at (b & 1, (b >> 1) & 1, (b >> 2) & 1)
in (x, y, z).  Edge e = 4 a + j lies along axis a; j = c_u + 2 c_v gives its
fixed coordinates on the other two axes (u, v) taken in increasing order.  A
corner bit is 1 ("inside") when A >= L.

Rule.  On every cube face whose edges cross the level:
  * two crossed edges: one segment joins them;
  * four crossed edges (inside corners on a diagonal): the inside corners are
    kept apart, i.e. each inside corner is cut off by the segment joining its
    two face edges.
Each segment is directed so that, seen from outside the cube (face normal
toward the viewer), the inside corners lie on its right.  Each crossed edge
then has one incoming and one outgoing segment, and the segments close into
loops.  Loops are listed by their lowest edge id and start there.  A loop
v0 v1 ... v(m-1) is fanned into triangles (v_s, v_(s+i), v_(s+i+1)) from the
first vertex v_s, in loop order, whose fan has no diagonal joining two
vertices that lie on a common cube face (such a diagonal would lie in that
face and be shared with the fan of the neighbouring cube, giving an edge
with four triangles).  With this direction the triangle normals
(right-hand rule) point from the inside corners to the outside ones.  The decision on a face depends on its four
corner bits only, so two cubes sharing the face agree and the mesh has no
cracks.
"""

import functools

import numpy as np

N_CORNERS = 8
N_EDGES = 12


def corner_pos(b):
    return (b & 1, (b >> 1) & 1, (b >> 2) & 1)


def _other_axes(a):
    return [c for c in range(3) if c != a]


def edge_corners(e):
    """Corner indices (lower, upper) of edge e."""
    a, j = divmod(e, 4)
    u, v = _other_axes(a)
    pos = [0, 0, 0]
    pos[u] = j & 1
    pos[v] = j >> 1
    c0 = pos[0] + 2 * pos[1] + 4 * pos[2]
    return c0, c0 + (1 << a)


def edge_axis(e):
    return e // 4


def edge_owner_offset(e):
    """Offset (x, y, z) of the node owning edge e (its lower corner) within the cell."""
    return corner_pos(edge_corners(e)[0])


def edge_mid2(e):
    """Twice the midpoint of edge e (integer coordinates)."""
    c0, c1 = edge_corners(e)
    p0, p1 = corner_pos(c0), corner_pos(c1)
    return tuple(p0[i] + p1[i] for i in range(3))


def faces():
    """List of (axis, side, corners in cyclic order, edges between them)."""
    out = []
    for a in range(3):
        u, v = _other_axes(a)
        for s in (0, 1):
            cyc = []
            for (cu, cv_) in ((0, 0), (1, 0), (1, 1), (0, 1)):
                pos = [0, 0, 0]
                pos[a], pos[u], pos[v] = s, cu, cv_
                cyc.append(pos[0] + 2 * pos[1] + 4 * pos[2])
            edges = []
            for i in range(4):
                ca, cb = cyc[i], cyc[(i + 1) % 4]
                e = _edge_between(ca, cb)
                edges.append(e)
            out.append((a, s, cyc, edges))
    return out


def _edge_between(ca, cb):
    for e in range(N_EDGES):
        if set(edge_corners(e)) == {ca, cb}:
            return e
    raise ValueError("corners are not adjacent")


def _cross(a, b):
    return (a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0])


def _orient(e_from, e_to, inside_corner, axis, side):
    """Direct the segment so the inside corner is on its right seen from outside."""
    p, q = edge_mid2(e_from), edge_mid2(e_to)
    c = tuple(2 * x for x in corner_pos(inside_corner))
    d = tuple(q[i] - p[i] for i in range(3))
    w = tuple(c[i] - p[i] for i in range(3))
    cr = _cross(d, w)
    normal = [0, 0, 0]
    normal[axis] = 1 if side == 1 else -1
    s = sum(cr[i] * normal[i] for i in range(3))
    if s == 0:
        raise AssertionError("degenerate orientation test")
    return (e_from, e_to) if s < 0 else (e_to, e_from)


def case_segments(case):
    """Directed segments (edge -> edge) of one case, from the face rule."""
    bit = [(case >> b) & 1 for b in range(N_CORNERS)]
    segs = []
    for (a, s, cyc, edges) in faces():
        crossed = [edges[i] for i in range(4) if bit[cyc[i]] != bit[cyc[(i + 1) % 4]]]
        if not crossed:
            continue
        if len(crossed) == 2:
            inside = [c for c in cyc if bit[c]]
            segs.append(_orient(crossed[0], crossed[1], inside[0], a, s))
        elif len(crossed) == 4:
            for i in range(4):
                if bit[cyc[i]]:
                    e_in, e_out = edges[(i - 1) % 4], edges[i]
                    segs.append(_orient(e_in, e_out, cyc[i], a, s))
        else:
            raise AssertionError("odd number of crossed edges on a face")
    return segs


def case_loops(case):
    """Closed loops of edge ids, each starting at its lowest id, ordered by it."""
    segs = case_segments(case)
    nxt = {}
    for p, q in segs:
        if p in nxt:
            raise AssertionError("edge with two outgoing segments")
        nxt[p] = q
    loops = []
    seen = set()
    for e in sorted(nxt):
        if e in seen:
            continue
        loop = [e]
        seen.add(e)
        cur = nxt[e]
        while cur != e:
            if cur in seen:
                raise AssertionError("loop does not close")
            loop.append(cur)
            seen.add(cur)
            cur = nxt[cur]
        loops.append(loop)
    return loops


def edge_faces(e):
    """The two cube faces (axis, side) that contain edge e."""
    return {(a, s) for (a, s, _, ed) in faces() if e in ed}


def _fan_ok(loop, s):
    m = len(loop)
    fa = edge_faces(loop[s])
    return all(not (fa & edge_faces(loop[(s + i) % m])) for i in range(2, m - 1))


def case_triangles(case):
    """Fan triangulation of every loop (see the module docstring for the start rule)."""
    tris = []
    for loop in case_loops(case):
        m = len(loop)
        s = next(k for k in range(m) if _fan_ok(loop, k))
        for i in range(1, m - 1):
            tris.append((loop[s], loop[(s + i) % m], loop[(s + i + 1) % m]))
    return tris


@functools.lru_cache(maxsize=None)
def table():
    """(n_tris[256] int, tris[256, max_tris, 3] int with -1 padding)."""
    all_tris = [case_triangles(c) for c in range(256)]
    mx = max(len(t) for t in all_tris)
    ntri = np.array([len(t) for t in all_tris], dtype=np.int64)
    tri = -np.ones((256, mx, 3), dtype=np.int64)
    for c, tl in enumerate(all_tris):
        for i, t in enumerate(tl):
            tri[c, i] = t
    return ntri, tri
