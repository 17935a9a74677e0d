"""Pins of the oracle's mesh rendering (Sec. III-C, III-E): coverage against
exact containment, depth against the analytic ray-plane hit, occlusion,
perspective-correct interpolation against a colour that is linear in 3D,
the multitexture blend against constant textures, and the silhouette of a
sphere against its analytic disc."""

from fractions import Fraction

import numpy as np
import pytest

from oracle import render

K = np.array([[100.0, 0.0, 50.0], [0.0, 100.0, 40.0], [0.0, 0.0, 1.0]], np.float32)
RT = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1).astype(np.float32)
W, H = 100, 80


def _at_pixel(u, v, z):
    """World point (camera = world) that projects to (u, v) at depth z."""
    return [(u - 50.0) / 100.0 * z, (v - 40.0) / 100.0 * z, z]


def test_coverage_is_exact_containment_and_depth_is_the_plane():
    z0 = 2.0
    uv = [(10.3, 5.7), (70.6, 20.2), (30.1, 66.4)]
    X = np.array([_at_pixel(u, v, z0) for u, v in uv], np.float32)
    depth, win = render.rasterise(X, [[0, 1, 2]], K, RT, W, H)
    u, v, _ = render.camera_project(K, RT, X)
    P = [(Fraction(float(a)), Fraction(float(b))) for a, b in zip(u, v)]

    def edge(a, b, px, py):
        return (b[0] - a[0]) * (py - a[1]) - (b[1] - a[1]) * (px - a[0])
    expect = np.zeros((H, W), bool)
    margin = []
    for j in range(H):
        for i in range(W):
            e = [edge(P[0], P[1], i, j), edge(P[1], P[2], i, j), edge(P[2], P[0], i, j)]
            expect[j, i] = all(x >= 0 for x in e) or all(x <= 0 for x in e)
            margin.append(min(abs(float(x)) for x in e))
    assert min(margin) > 1e-3                     # no pixel centre on an edge: containment is robust
    assert np.array_equal(win >= 0, expect) and expect.sum() > 500
    assert np.all(depth[expect] == np.float32(z0)) and np.all(depth[~expect] == 0)


def test_tilted_plane_depth_is_the_ray_plane_intersection():
    # plane z = 2 + 0.3 x - 0.2 y, a quad covering the whole view
    def on_plane(u, v):
        dx, dy = (u - 50.0) / 100.0, (v - 40.0) / 100.0
        z = 2.0 / (1.0 - 0.3 * dx + 0.2 * dy)
        return [dx * z, dy * z, z]
    X = np.array([on_plane(-5, -5), on_plane(105, -5), on_plane(105, 85), on_plane(-5, 85)], np.float32)
    depth, win = render.rasterise(X, [[0, 1, 2], [0, 2, 3]], K, RT, W, H)
    assert np.all(win >= 0)
    # the float32 vertices define the plane: fit it exactly through them
    Xd = X.astype(np.float64)
    n = np.cross(Xd[1] - Xd[0], Xd[2] - Xd[0])
    jj, ii = np.mgrid[0:H, 0:W]
    ray = np.stack([(ii - 50.0) / 100.0, (jj - 40.0) / 100.0, np.ones_like(ii, float)], -1)
    z = (n @ Xd[0]) / (ray @ n)
    assert np.max(np.abs(depth - z) / z) < 2e-7


def test_nearest_surface_wins_whatever_the_order():
    a = [_at_pixel(u, v, 2.0) for u, v in [(5.5, 5.5), (90.5, 10.5), (40.5, 70.5)]]
    b = [_at_pixel(u, v, 3.0) for u, v in [(10.5, 2.5), (95.5, 40.5), (20.5, 75.5)]]
    X = np.array(a + b, np.float32)
    d1, w1 = render.rasterise(X, [[0, 1, 2], [3, 4, 5]], K, RT, W, H)
    d2, w2 = render.rasterise(X, [[3, 4, 5], [0, 1, 2]], K, RT, W, H)
    assert np.array_equal(d1, d2)
    both = (w1 >= 0)
    near = render.rasterise(X, [[0, 1, 2]], K, RT, W, H)[1] >= 0
    assert np.all(d1[near] == np.float32(2.0)) and np.all(d1[both & ~near] == np.float32(3.0))
    # exact tie: the lower triangle index wins
    d3, w3 = render.rasterise(X[:3], [[0, 1, 2], [0, 1, 2]], K, RT, W, H)
    assert np.all(w3[w3 >= 0] == 0)


def test_triangles_behind_the_near_plane_are_not_drawn():
    X = np.array([[0.0, 0.0, -0.5], [0.3, 0.0, 2.0], [0.0, 0.3, 2.0]], np.float32)
    depth, win = render.rasterise(X, [[0, 1, 2]], K, RT, W, H)
    assert not np.any(win >= 0)
    X[0, 2] = 2 * render.Z_NEAR
    assert np.any(render.rasterise(X, [[0, 1, 2]], K, RT, W, H)[1] >= 0)


def test_vertex_colour_is_perspective_correct():
    # a steeply tilted triangle; colour linear in 3D: c(X) = 20 + 50 (X.e - 0.77)
    X = np.array([[-0.8, -0.6, 1.5], [0.9, -0.5, 4.5], [0.0, 0.8, 2.5]], np.float32)

    def colour(P):
        return 20.0 + 50.0 * (np.asarray(P, np.float64) @ np.array([0.5, 0.8, 1.1]) - 0.77)
    cv = np.stack([colour(X)] * 3, axis=1)
    assert cv.min() > 0 and cv.max() < 255
    depth, rgb = render.render_vertex_colour(X, [[0, 1, 2]], cv, K, RT, W, H)
    jj, ii = np.nonzero(depth > 0)
    assert len(jj) > 500
    P = np.stack([(ii - 50.0) / 100.0, (jj - 40.0) / 100.0, np.ones(len(ii))], 1) * depth[jj, ii, None]
    want = np.floor(colour(P) + 0.5)
    assert np.max(np.abs(rgb[jj, ii, 0].astype(float) - want)) <= 1
    # screen-affine interpolation would be visibly off on this triangle
    u, v, _ = render.camera_project(K, RT, X)
    T = np.array([[u[1] - u[0], u[2] - u[0]], [v[1] - v[0], v[2] - v[0]]])
    ab = np.linalg.solve(T, np.stack([ii - u[0], jj - v[0]]))
    affine = (1 - ab[0] - ab[1]) * cv[0, 0] + ab[0] * cv[1, 0] + ab[1] * cv[2, 0]
    assert np.max(np.abs(affine - want)) > 5


def test_multitexture_blend_of_constant_views():
    X = np.array([_at_pixel(u, v, 2.0) for u, v in [(5.5, 5.5), (90.5, 10.5), (40.5, 70.5)]], np.float32)
    views = [{"rgb": np.full((30, 40, 3), (200, 10, 30), np.uint8)},
             {"rgb": np.full((30, 40, 3), (0, 250, 90), np.uint8)},
             {"rgb": np.full((30, 40, 3), (255, 255, 255), np.uint8)}]
    wts = np.array([[0.25, 0.75, 0.5]] * 3)
    wts[1, 2] = 0.0                         # view 2 is not visible at one vertex: skipped
    uv = np.full((3, 3, 2), 10.0)
    depth, rgb = render.render_multitexture(X, [[0, 1, 2]], wts, uv, views, K, RT, W, H)
    want = np.floor((0.25 * np.array([200, 10, 30]) + 0.75 * np.array([0, 250, 90])) + 0.5)
    drawn = depth > 0
    assert drawn.sum() > 500 and np.all(rgb[drawn] == want) and np.all(rgb[~drawn] == 0)
    # no view weighted at all three vertices: black
    wts[:, :] = 0.0
    wts[0, :] = 1.0
    _, rgb0 = render.render_multitexture(X, [[0, 1, 2]], wts, uv, views, K, RT, W, H)
    assert np.all(rgb0 == 0)


@pytest.mark.parametrize("D", [2.5, 4.0])
def test_sphere_silhouette_is_the_analytic_disc(D):
    r = 0.6
    th, ph = np.meshgrid(np.linspace(0, np.pi, 97), np.linspace(0, 2 * np.pi, 193), indexing="ij")
    P = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], -1).reshape(-1, 3) * r
    P[:, 2] += D
    nt, nph = th.shape
    tris = []
    for a in range(nt - 1):
        for b in range(nph - 1):
            i0, i1, i2, i3 = a * nph + b, a * nph + b + 1, (a + 1) * nph + b, (a + 1) * nph + b + 1
            tris += [[i0, i2, i1], [i1, i2, i3]]
    Kb = np.array([[300.0, 0, 160.0], [0, 300.0, 120.0], [0, 0, 1.0]], np.float32)
    depth, _ = render.rasterise(P.astype(np.float32), tris, Kb, RT, 320, 240)
    area = (depth > 0).sum()
    rad = 300.0 * r / np.sqrt(D * D - r * r)        # image radius of the sphere's outline
    assert abs(area - np.pi * rad * rad) / (np.pi * rad * rad) < 0.02
    assert abs(depth[120, 160] - (D - r)) < 1e-3
