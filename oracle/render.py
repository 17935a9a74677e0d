"""Rendering a triangle mesh into a planar view (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. III-E evaluates a reconstruction by projecting the mesh into the K + K'
sensor views and reading back the depth and colour buffers; Sec. III-C
renders every triangle with the per-vertex weights and UVs (multitexture
blending), and Sec. V compares that with a colour-per-vertex rendering
(Fig. 19).  The paper uses OpenGL for both; here the depth and colour
buffers are defined directly.

Readings (float64 unless stated; the operation order below is part of the
definition, because the coverage and the nearest-surface choice are
decisions taken on rounded numbers):

* camera: x_c = R X + t, each row summed as ((r0 X + r1 Y) + r2 Z) + t_r;
  a = x_c/z_c, b = y_c/z_c, u = (K00 a + K01 b) + K02, v = K11 b + K12;
  pixel (i, j) is the sample point (u, v) = (i, j);
* a triangle is skipped when a vertex has z_c < Z_NEAR or when its screen
  area (ub-ua)(vc-va) - (vb-va)(uc-ua) is 0 (or not finite);
* a pixel is covered iff its three edge functions
  e_ab = (ub-ua)(py-va) - (vb-va)(px-ua) (and cyclic) are all >= 0 or all
  <= 0 (no face culling; pixels on an edge belong to both triangles);
* its depth is the camera z of the point where the pixel's ray
  d = (dx, dy, 1), dy = (py - K12)/K11, dx = ((px - K02) - K01 dy)/K00,
  meets the triangle's plane: n = (B - A) x (C - A) in camera coordinates,
  z = ((nx Ax + ny Ay) + nz Az) / ((nx dx + ny dy) + nz); kept iff the
  denominator is not 0 and z > 0;
* the nearest surface wins: the smallest (float32(z), triangle index) pair;
  the depth buffer holds float32(z), 0 where nothing is drawn;
* colours interpolate with the perspective-correct barycentrics of the hit
  point P = z d: lambda_A = n.((B - P) x (C - P)) / n.n (and cyclic);
  colour-per-vertex: c = sum lambda_i c_i; multitexture: for every view k
  whose weight is > 0 at all three vertices, w_k = sum lambda_i w_k,i and
  uv_k = sum lambda_i uv_k,i, c = sum_k w_k RGB_k(uv_k) / sum_k w_k with the
  clamped bilinear sample of ``oracle.texture``; stored as floor(c + 1/2)
  in u8, 0 where nothing is drawn or no view applies.
"""

import numpy as np

from oracle.texture import bilinear_rgb

Z_NEAR = 0.01          # metres: triangles with a vertex closer to the camera plane are not drawn


def camera_project(K, world_to_cam, X):
    """(u, v, x_c [n, 3]) of world points X in the stated operation order."""
    K = np.asarray(K, dtype=np.float32).astype(np.float64).reshape(3, 3)
    RT = np.asarray(world_to_cam, dtype=np.float32).astype(np.float64).reshape(3, 4)
    X = np.asarray(X, dtype=np.float32).astype(np.float64)
    xc = np.empty_like(X)
    for r in range(3):
        xc[:, r] = ((RT[r, 0] * X[:, 0] + RT[r, 1] * X[:, 1]) + RT[r, 2] * X[:, 2]) + RT[r, 3]
    with np.errstate(divide="ignore", invalid="ignore"):
        a = xc[:, 0] / xc[:, 2]
        b = xc[:, 1] / xc[:, 2]
    u = (K[0, 0] * a + K[0, 1] * b) + K[0, 2]
    v = K[1, 1] * b + K[1, 2]
    return u, v, xc


def pixel_ray(K, px, py):
    """Ray (dx, dy, 1) through pixel centres (px, py) (float64 arrays)."""
    K = np.asarray(K, dtype=np.float32).astype(np.float64).reshape(3, 3)
    dy = (py - K[1, 2]) / K[1, 1]
    dx = ((px - K[0, 2]) - K[0, 1] * dy) / K[0, 0]
    return dx, dy


def rasterise(vertices, tris, K, world_to_cam, w, h):
    """Depth buffer [h, w] float32 and the winning triangle [h, w] int64 (-1 = none)."""
    tris = np.asarray(tris, dtype=np.int64).reshape(-1, 3)
    depth = np.zeros((h, w), np.float32)
    winner = -np.ones((h, w), np.int64)
    if len(tris) == 0:
        return depth, winner
    u, v, xc = camera_project(K, world_to_cam, vertices)
    ia, ib, ic = tris[:, 0], tris[:, 1], tris[:, 2]
    ua, ub, uc = u[ia], u[ib], u[ic]
    va, vb, vc = v[ia], v[ib], v[ic]
    with np.errstate(invalid="ignore"):
        front = (xc[ia, 2] >= Z_NEAR) & (xc[ib, 2] >= Z_NEAR) & (xc[ic, 2] >= Z_NEAR)
        area = (ub - ua) * (vc - va) - (vb - va) * (uc - ua)
        ok = front & np.isfinite(area) & (area != 0.0)
        x0 = np.maximum(np.ceil(np.minimum(np.minimum(ua, ub), uc)), 0.0)
        x1 = np.minimum(np.floor(np.maximum(np.maximum(ua, ub), uc)), w - 1.0)
        y0 = np.maximum(np.ceil(np.minimum(np.minimum(va, vb), vc)), 0.0)
        y1 = np.minimum(np.floor(np.maximum(np.maximum(va, vb), vc)), h - 1.0)
    ok &= (x1 >= x0) & (y1 >= y0)
    t_ok = np.nonzero(ok)[0]
    nx_ = (x1[t_ok] - x0[t_ok] + 1).astype(np.int64)
    ny_ = (y1[t_ok] - y0[t_ok] + 1).astype(np.int64)
    cnt = nx_ * ny_
    # one candidate per (triangle, pixel of its bounding box)
    t = np.repeat(t_ok, cnt)
    first = np.repeat(np.cumsum(cnt) - cnt, cnt)
    local = np.arange(len(t)) - first
    rep_nx = np.repeat(nx_, cnt)
    px = x0[t] + (local % rep_nx)
    py = y0[t] + (local // rep_nx)
    ua, ub, uc, va, vb, vc = ua[t], ub[t], uc[t], va[t], vb[t], vc[t]
    e0 = (ub - ua) * (py - va) - (vb - va) * (px - ua)
    e1 = (uc - ub) * (py - vb) - (vc - vb) * (px - ub)
    e2 = (ua - uc) * (py - vc) - (va - vc) * (px - uc)
    inside = ((e0 >= 0) & (e1 >= 0) & (e2 >= 0)) | ((e0 <= 0) & (e1 <= 0) & (e2 <= 0))
    t, px, py = t[inside], px[inside], py[inside]
    A, B, C = xc[ia[t]], xc[ib[t]], xc[ic[t]]
    e1v = B - A
    e2v = C - A
    nx = e1v[:, 1] * e2v[:, 2] - e1v[:, 2] * e2v[:, 1]
    ny = e1v[:, 2] * e2v[:, 0] - e1v[:, 0] * e2v[:, 2]
    nz = e1v[:, 0] * e2v[:, 1] - e1v[:, 1] * e2v[:, 0]
    num = (nx * A[:, 0] + ny * A[:, 1]) + nz * A[:, 2]
    dx, dy = pixel_ray(K, px, py)
    den = (nx * dx + ny * dy) + nz
    with np.errstate(divide="ignore", invalid="ignore"):
        z = num / den
        keep = (den != 0.0) & (z > 0.0) & np.isfinite(z)
    t, px, py, z = t[keep], px[keep], py[keep], z[keep].astype(np.float32)
    pix = py.astype(np.int64) * w + px.astype(np.int64)
    # nearest surface: smallest (z, triangle) per pixel
    order = np.lexsort((t, z, pix))
    pix, t, z = pix[order], t[order], z[order]
    head = np.ones(len(pix), bool)
    head[1:] = pix[1:] != pix[:-1]
    depth.reshape(-1)[pix[head]] = z[head]
    winner.reshape(-1)[pix[head]] = t[head]
    return depth, winner


def barycentrics(vertices, tris, K, world_to_cam, depth, winner):
    """Perspective-correct barycentrics [h, w, 3] of each drawn pixel (0 elsewhere)."""
    h, w = depth.shape
    lam = np.zeros((h, w, 3))
    jj, ii = np.nonzero(winner >= 0)
    if len(jj) == 0:
        return lam
    tris = np.asarray(tris, dtype=np.int64).reshape(-1, 3)
    _, _, xc = camera_project(K, world_to_cam, vertices)
    tri = tris[winner[jj, ii]]
    A, B, C = xc[tri[:, 0]], xc[tri[:, 1]], xc[tri[:, 2]]
    dx, dy = pixel_ray(K, ii.astype(np.float64), jj.astype(np.float64))
    z = depth[jj, ii].astype(np.float64)
    P = np.stack([z * dx, z * dy, z], axis=1)
    n = np.cross(B - A, C - A)
    nn = (n * n).sum(1)
    la = (n * np.cross(B - P, C - P)).sum(1) / nn
    lb = (n * np.cross(C - P, A - P)).sum(1) / nn
    lc = (n * np.cross(A - P, B - P)).sum(1) / nn
    lam[jj, ii] = np.stack([la, lb, lc], axis=1)
    return lam


def _to_u8(c):
    return np.clip(np.floor(c + 0.5), 0, 255).astype(np.uint8)


def render_vertex_colour(vertices, tris, vertex_rgb, K, world_to_cam, w, h):
    """(depth [h, w] f32, rgb [h, w, 3] u8) with colours interpolated per pixel."""
    depth, winner = rasterise(vertices, tris, K, world_to_cam, w, h)
    lam = barycentrics(vertices, tris, K, world_to_cam, depth, winner)
    rgb = np.zeros((h, w, 3), np.uint8)
    jj, ii = np.nonzero(winner >= 0)
    if len(jj):
        tri = np.asarray(tris, dtype=np.int64).reshape(-1, 3)[winner[jj, ii]]
        col = np.asarray(vertex_rgb, dtype=np.float64)
        c = sum(lam[jj, ii, m, None] * col[tri[:, m]] for m in range(3))
        rgb[jj, ii] = _to_u8(c)
    return depth, rgb


def render_multitexture(vertices, tris, weights, uv, views, K, world_to_cam, w, h):
    """(depth, rgb u8) blending the views' RGB images with the per-vertex
    weights [V, k] and UVs [V, k, 2] interpolated across each triangle."""
    depth, winner = rasterise(vertices, tris, K, world_to_cam, w, h)
    lam = barycentrics(vertices, tris, K, world_to_cam, depth, winner)
    rgb = np.zeros((h, w, 3), np.uint8)
    jj, ii = np.nonzero(winner >= 0)
    if len(jj) == 0:
        return depth, rgb
    tri = np.asarray(tris, dtype=np.int64).reshape(-1, 3)[winner[jj, ii]]
    L = lam[jj, ii]
    W = np.asarray(weights, dtype=np.float64)
    UV = np.asarray(uv, dtype=np.float64)
    acc = np.zeros((len(jj), 3))
    wsum = np.zeros(len(jj))
    for k, vw in enumerate(views):
        wv = W[tri, k]                                   # [n, 3]
        use = (wv > 0).all(axis=1)
        if not np.any(use):
            continue
        wk = (L[use] * wv[use]).sum(1)
        uk = (L[use] * UV[tri[use], k, 0]).sum(1)
        vk = (L[use] * UV[tri[use], k, 1]).sum(1)
        acc[use] += wk[:, None] * bilinear_rgb(np.asarray(vw["rgb"]), uk, vk)
        wsum[use] += wk
    out = np.zeros((len(jj), 3))
    good = wsum > 0
    out[good] = acc[good] / wsum[good, None]
    rgb[jj, ii] = _to_u8(out)
    return depth, rgb
