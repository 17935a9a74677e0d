"""Per-vertex texture mapping (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. III-C: for a vertex X, V(X) is the set of depth cameras in which X is
visible; for k in V(X), u_k = Pi_k(X) is its depth pixel and u_k^RGB =
Pi_k^RGB(X) its RGB (UV) coordinate; each vertex carries the weights W_k(u_k)
and the UVs; visibility in the RGB camera is taken equal to visibility in
its depth camera.  The paper then blends the textures with OpenGL; no
graphics stack is used here, and the blend is restated per vertex.

Readings (all in float64):
* camera model: x_c = R X + t (``world_to_cam`` is [R | t], 3x4 row-major),
  (u', v', w') = K x_c, u = u'/w', v = v'/w'; pixel (i, j) is centred at
  integer coordinates; x_c.z <= 0 is not visible;
* nearest pixel floor(u + 1/2), floor(v + 1/2); visible iff inside the image,
  D > 0 there (foreground) and |D - x_c.z| <= tau;
* w_k = W_k at that nearest depth pixel (0 when not visible), and also 0 when
  the RGB projection falls outside [0, w-1] x [0, h-1];
* uv_k = (u_rgb, v_rgb) in RGB pixels, (-1, -1) when w_k = 0;
* colour c = sum_k w_k RGB_k(uv_k) / sum_k w_k with bilinear RGB samples,
  stored as floor(c + 1/2) in u8; ``textured`` = (sum_k w_k > 0).
"""

import numpy as np


def project(K, world_to_cam, X):
    """Return (u, v, z_cam) for points X [n, 3] (float64)."""
    K = np.asarray(K, dtype=np.float64).reshape(3, 3)
    RT = np.asarray(world_to_cam, dtype=np.float64).reshape(3, 4)
    xc = X @ RT[:, :3].T + RT[:, 3]
    uvw = xc @ K.T
    with np.errstate(divide="ignore", invalid="ignore"):
        u = uvw[:, 0] / uvw[:, 2]
        v = uvw[:, 1] / uvw[:, 2]
    return u, v, xc[:, 2]


def bilinear_rgb(img, u, v):
    """Bilinear RGB at continuous pixel coordinates (clamped), float64 [n, 3]."""
    h, w = img.shape[:2]
    x0 = np.floor(u).astype(np.int64)
    y0 = np.floor(v).astype(np.int64)
    fx = u - x0
    fy = v - y0
    xa = np.clip(x0, 0, w - 1)
    xb = np.clip(x0 + 1, 0, w - 1)
    ya = np.clip(y0, 0, h - 1)
    yb = np.clip(y0 + 1, 0, h - 1)
    im = img.astype(np.float64)
    c00 = im[ya, xa]
    c10 = im[ya, xb]
    c01 = im[yb, xa]
    c11 = im[yb, xb]
    return ((1 - fx)[:, None] * (1 - fy)[:, None] * c00 + fx[:, None] * (1 - fy)[:, None] * c10
            + (1 - fx)[:, None] * fy[:, None] * c01 + fx[:, None] * fy[:, None] * c11)


def texture(vertices, views, depth_tol):
    """Per-vertex weights [V, K], uv [V, K, 2], rgb [V, 3] u8, textured [V] u8."""
    X = np.asarray(vertices, dtype=np.float64)
    nv = len(X)
    K = len(views)
    weights = np.zeros((nv, K))
    uv = -np.ones((nv, K, 2))
    acc = np.zeros((nv, 3))
    wsum = np.zeros(nv)
    for k, vw in enumerate(views):
        depth = np.asarray(vw["depth"], dtype=np.float64)
        conf = np.asarray(vw["conf"], dtype=np.float64)
        h, w = depth.shape
        u, v, z = project(vw["K"], vw["world_to_cam"], X)
        with np.errstate(invalid="ignore"):
            px = np.floor(u + 0.5)
            py = np.floor(v + 0.5)
            inside = (z > 0) & (px >= 0) & (px < w) & (py >= 0) & (py < h)
        pxi = np.where(inside, px, 0).astype(np.int64)
        pyi = np.where(inside, py, 0).astype(np.int64)
        D = depth[pyi, pxi]
        vis = inside & (D > 0) & (np.abs(D - z) <= depth_tol)
        wk = np.where(vis, conf[pyi, pxi], 0.0)
        rgb = np.asarray(vw["rgb"])
        rh, rw = rgb.shape[:2]
        ur, vr, zr = project(vw["K_rgb"], vw["world_to_rgb"], X)
        with np.errstate(invalid="ignore"):
            in_rgb = (zr > 0) & (ur >= 0) & (ur <= rw - 1) & (vr >= 0) & (vr <= rh - 1)
        wk = np.where(in_rgb, wk, 0.0)
        use = wk > 0
        weights[:, k] = wk
        uv[use, k, 0] = ur[use]
        uv[use, k, 1] = vr[use]
        if np.any(use):
            acc[use] += wk[use, None] * bilinear_rgb(rgb, ur[use], vr[use])
        wsum += wk
    textured = wsum > 0
    col = np.zeros((nv, 3))
    col[textured] = acc[textured] / wsum[textured, None]
    rgb_out = np.clip(np.floor(col + 0.5), 0, 255).astype(np.uint8)
    return {"weights": weights, "uv": uv, "rgb": rgb_out, "textured": textured.astype(np.uint8)}
