"""The whole per-frame reconstruction path in the paper's order (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. III-B then III-C: splat eq.(1)(2) -> forward 3D FFT of each component
-> integration filter -> inverse 3D FFT -> level L -> marching cubes ->
per-vertex texture.
"""

import time

from . import conventions as cv
from . import splat as osplat
from . import spectral, level, mc, texture


def default_depth_tol(grid_n, bbox):
    """tau = max(3 h_max, 0.02 m): the visibility tolerance (not in the paper)."""
    h = cv.voxel_size(grid_n, bbox)
    return max(3.0 * max(h), 0.02)


def reconstruct(points, normals, weights, grid_n, bbox, mode=cv.SPLAT_WEIGHTED,
                views=None, depth_tol=None, timings=None):
    """Run the oracle path; returns dict(V, A, L, mesh, tex)."""
    t = {}
    t0 = time.perf_counter()
    V = osplat.splat(points, normals, weights, grid_n, bbox, mode=mode)
    t["splat"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    A = spectral.integrate(V, grid_n, bbox)
    t["fft"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    L = level.iso_level(A, points, grid_n, bbox)
    t["level"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    mesh = mc.marching_cubes(A, L, grid_n, bbox)
    t["mc"] = time.perf_counter() - t0
    tex = None
    if views:
        t0 = time.perf_counter()
        tol = default_depth_tol(grid_n, bbox) if depth_tol is None else depth_tol
        tex = texture.texture(mesh["vertices"], views, tol)
        t["texture"] = time.perf_counter() - t0
    if timings is not None:
        timings.update(t)
    return {"V": V, "A": A, "L": L, "mesh": mesh, "tex": tex}
