"""Raw reconstruction of oriented, weighted points from depth maps (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. III-A, per depth camera k and foreground pixel u (D_k(u) > 0):

* the 3D point X_k(u) = Pi_k^-1(u, D_k(u)): camera coordinates
  ((u_x - c_x) / f_x * D, (u_y - c_y) / f_y * D, D), world X = R^T (x_c - t)
  for world_to_cam = [R | t];
* the normal N_k(u) from an organised triangulation of the pixel grid: every
  2 x 2 pixel quad with top-left (row j, column i) gives the triangles
  (p[j,i], p[j,i+1], p[j+1,i]) and (p[j,i+1], p[j+1,i+1], p[j+1,i]); a
  triangle is kept iff its three pixels are foreground, its largest corner
  depth difference is within the discontinuity threshold
  (``conventions.TSDC_STEP`` + 3 ``TSDC_NOISE`` z_max^2) and its area is not
  zero; its unit normal is oriented toward the camera (n . centroid < 0 in
  camera coordinates); the vertex normal is the normalised sum of the unit
  normals of the kept triangles that contain the pixel;
* the confidence W = W1 W2 with W1 = max(<-x_c / |x_c|, N>, 0) and W2 the
  mean of the binary silhouette over a (2 r + 1)^2 window (r =
  ``conventions.W2_RADIUS``), zero outside the image.

A pixel gives a point iff it is foreground and at least one kept triangle
contains it (the sum of its normals is not zero).  Points are listed in
row-major pixel order.  Inputs are the float32 depth map and camera that the
kernels receive, promoted to float64.
"""

import numpy as np

from . import conventions as cv


def camera_points(depth, K):
    """x_c per pixel [h, w, 3] (float64) of a depth map (0 = background)."""
    D = np.asarray(depth, dtype=np.float64)
    K = np.asarray(K, dtype=np.float64)
    h, w = D.shape
    v, u = np.meshgrid(np.arange(h, dtype=np.float64), np.arange(w, dtype=np.float64), indexing="ij")
    return np.stack([(u - K[0, 2]) / K[0, 0] * D, (v - K[1, 2]) / K[1, 1] * D, D], axis=-1)


def triangle_normals(xc, depth, step=cv.TSDC_STEP, noise=cv.TSDC_NOISE):
    """Kept flags and camera-facing unit normals of the two triangle families.

    Returns [(corners, keep [h-1, w-1], n [h-1, w-1, 3])] for the triangles
    (00, 01, 10) and (01, 11, 10) of every quad, corners as (dj, di) offsets.
    """
    D = np.asarray(depth, dtype=np.float64)
    fg = D > 0
    out = []
    for corners in (((0, 0), (0, 1), (1, 0)), ((0, 1), (1, 1), (1, 0))):
        P = [xc[a:a + xc.shape[0] - 1, b:b + xc.shape[1] - 1] for (a, b) in corners]
        Z = [D[a:a + D.shape[0] - 1, b:b + D.shape[1] - 1] for (a, b) in corners]
        F = [fg[a:a + fg.shape[0] - 1, b:b + fg.shape[1] - 1] for (a, b) in corners]
        zmax = np.maximum(np.maximum(Z[0], Z[1]), Z[2])
        dz = np.maximum(np.maximum(np.abs(Z[0] - Z[1]), np.abs(Z[1] - Z[2])), np.abs(Z[0] - Z[2]))
        n = np.cross(P[1] - P[0], P[2] - P[0])
        ln = np.linalg.norm(n, axis=-1)
        keep = F[0] & F[1] & F[2] & (dz <= step + 3.0 * noise * zmax * zmax) & (ln > 0)
        n = n / np.where(ln > 0, ln, 1.0)[..., None]
        centroid = (P[0] + P[1] + P[2]) / 3.0
        n = np.where((np.sum(n * centroid, axis=-1) > 0)[..., None], -n, n)
        out.append((corners, keep, np.where(keep[..., None], n, 0.0)))
    return out


def vertex_normals(xc, depth, step=cv.TSDC_STEP, noise=cv.TSDC_NOISE):
    """Camera-space unit vertex normals [h, w, 3] and the point mask [h, w]."""
    D = np.asarray(depth, dtype=np.float64)
    h, w = D.shape
    acc = np.zeros((h, w, 3))
    for corners, keep, n in triangle_normals(xc, D, step, noise):
        for (a, b) in corners:
            acc[a:a + h - 1, b:b + w - 1] += n
    ln = np.linalg.norm(acc, axis=-1)
    mask = (D > 0) & (ln > 0)
    return np.where(mask[..., None], acc / np.where(ln > 0, ln, 1.0)[..., None], 0.0), mask


def silhouette_mean(depth, radius=cv.W2_RADIUS):
    """W2: mean of (D > 0) over the (2r+1)^2 window around each pixel, zero outside."""
    m = (np.asarray(depth) > 0).astype(np.float64)
    h, w = m.shape
    k = 2 * radius + 1
    padded = np.zeros((h + 2 * radius, w + 2 * radius))
    padded[radius:radius + h, radius:radius + w] = m
    out = np.zeros((h, w))
    for dj in range(k):
        for di in range(k):
            out += padded[dj:dj + h, di:di + w]
    return out / (k * k)


def raw_points(depth, K, world_to_cam, step=cv.TSDC_STEP, noise=cv.TSDC_NOISE, radius=cv.W2_RADIUS):
    """Points, normals (world), weights W = W1 W2 of one depth map, row-major
    pixel order, and the per-pixel confidence map (0 where no point)."""
    xc = camera_points(depth, K)
    nc, mask = vertex_normals(xc, depth, step, noise)
    ln = np.linalg.norm(xc, axis=-1)
    xhat = -xc / np.where(ln > 0, ln, 1.0)[..., None]
    w1 = np.maximum(np.sum(xhat * nc, axis=-1), 0.0)
    W = np.where(mask, w1 * silhouette_mean(depth, radius), 0.0)
    RT = np.asarray(world_to_cam, dtype=np.float64)
    R, t = RT[:, :3], RT[:, 3]
    Xw = (xc - t) @ R              # R^T (x_c - t) per row vector
    Nw = nc @ R                    # R^T n
    return Xw[mask], Nw[mask], W[mask], W
