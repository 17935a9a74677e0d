"""Splatting of oriented points into the gradient field V (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Follows Sec. III-B, eq. (1) and eq. (2):

  U(q) = sum_i g(|X_i - p(q)|; sigma1) W_i N_i
  d(q) = sum_i g(|X_i - p(q)|; sigma2) W_i,      g(x; s) = s^-1 exp(-x^2/s^2)
  V(q) = U(q) / d(q)     (w_k(u, q) = W_k(u) / d(q) with d depending on q only)

summed in float64 over the 4^3 nodes around each accepted point, in point
order.  V = 0 where d = 0.  The simple (non-weighted) variant of the same
section snaps each point to its nearest node and divides by the count.
"""

import numpy as np

from . import conventions as cv


def node_coords(points, grid_n, bbox):
    """Continuous node coordinate t = (X - b_min)/h - 1/2 per axis (float64)."""
    p = np.asarray(points, dtype=np.float64)
    h = np.array(cv.voxel_size(grid_n, bbox))
    bmin = np.array([float(b) for b in bbox[:3]])
    return (p - bmin) / h - 0.5


def accepted_mask(points, grid_n, bbox):
    """A point is accepted iff 1 <= t_c < n_c - 2 on every axis (stencil inside)."""
    t = node_coords(points, grid_n, bbox)
    n = np.array(grid_n, dtype=np.float64)
    ok = np.all((t >= 1.0) & (t < n - 2.0), axis=1)
    return ok & np.all(np.isfinite(t), axis=1)


def node_position(q, grid_n, bbox):
    """p(q) = b_min + (q + 1/2) h for integer node indices q[..., 3] (x, y, z)."""
    h = np.array(cv.voxel_size(grid_n, bbox))
    bmin = np.array([float(b) for b in bbox[:3]])
    return bmin + (np.asarray(q, dtype=np.float64) + 0.5) * h


def _flat(q, grid_n):
    nx, ny, _ = (int(v) for v in grid_n)
    return q[..., 0] + nx * (q[..., 1] + ny * q[..., 2])


def splat_weighted(points, normals, weights, grid_n, bbox, sigma1_scale=1.0,
                   sigma2_ratio2=cv.SIGMA2_RATIO2, return_ud=False):
    """Eq. (1)-(2): returns V as float64 [3, nz, ny, nx] (and U, d if asked)."""
    nx, ny, nz = (int(v) for v in grid_n)
    pts = np.asarray(points, dtype=np.float64)
    nrm = np.asarray(normals, dtype=np.float64)
    w = np.ones(len(pts)) if weights is None else np.asarray(weights, dtype=np.float64)
    ok = accepted_mask(pts, grid_n, bbox)
    pts, nrm, w = pts[ok], nrm[ok], w[ok]
    s1, s2 = cv.sigmas(grid_n, bbox, sigma1_scale, sigma2_ratio2)
    t = node_coords(pts, grid_n, bbox)
    base = np.floor(t).astype(np.int64) - cv.STENCIL_LO
    m = nx * ny * nz
    U = np.zeros((3, m))
    d = np.zeros(m)
    for oz in range(cv.STENCIL):
        for oy in range(cv.STENCIL):
            for ox in range(cv.STENCIL):
                q = base + np.array([ox, oy, oz])
                r2 = np.sum((pts - node_position(q, grid_n, bbox)) ** 2, axis=1)
                g1 = np.exp(-r2 / s1 ** 2) / s1
                g2 = np.exp(-r2 / s2 ** 2) / s2
                f = _flat(q, grid_n)
                for c in range(3):
                    np.add.at(U[c], f, g1 * w * nrm[:, c])
                np.add.at(d, f, g2 * w)
    V = np.zeros_like(U)
    pos = d > 0
    V[:, pos] = U[:, pos] / d[pos]
    V = V.reshape(3, nz, ny, nx)
    if return_ud:
        return V, U.reshape(3, nz, ny, nx), d.reshape(nz, ny, nx)
    return V


def splat_simple(points, normals, grid_n, bbox):
    """Simple variant: nearest node floor(t + 1/2), mean of N per node, W ignored."""
    nx, ny, nz = (int(v) for v in grid_n)
    pts = np.asarray(points, dtype=np.float64)
    nrm = np.asarray(normals, dtype=np.float64)
    ok = accepted_mask(pts, grid_n, bbox)
    pts, nrm = pts[ok], nrm[ok]
    q = np.floor(node_coords(pts, grid_n, bbox) + 0.5).astype(np.int64)
    f = _flat(q, grid_n)
    m = nx * ny * nz
    U = np.zeros((3, m))
    cnt = np.zeros(m)
    for c in range(3):
        np.add.at(U[c], f, nrm[:, c])
    np.add.at(cnt, f, 1.0)
    V = np.zeros_like(U)
    pos = cnt > 0
    V[:, pos] = U[:, pos] / cnt[pos]
    return V.reshape(3, nz, ny, nx)


def splat(points, normals, weights, grid_n, bbox, mode=cv.SPLAT_WEIGHTED, **kw):
    """Dispatch on the splat mode of Sec. III-B (weighted eq.(1)(2) or simple)."""
    if mode == cv.SPLAT_WEIGHTED:
        return splat_weighted(points, normals, weights, grid_n, bbox, **kw)
    if mode == cv.SPLAT_SIMPLE:
        return splat_simple(points, normals, grid_n, bbox)
    raise ValueError(f"unknown splat mode {mode}")
