"""Pins for the oracle iso-level (Sec. III-B: L = mean of A at the samples), no GPU."""

import numpy as np

from oracle import conventions as cv
from oracle import level, splat as S

GRID = (10, 12, 9)
BBOX = (-0.5, 0.0, -1.0, 0.5, 1.2, 0.8)


def _nodes(grid_n, bbox):
    h = cv.voxel_size(grid_n, bbox)
    nx, ny, nz = grid_n
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return (bbox[0] + (x + 0.5) * h[0], bbox[1] + (y + 0.5) * h[1], bbox[2] + (z + 0.5) * h[2])


def test_linear_field_is_reproduced():
    X, Y, Z = _nodes(GRID, BBOX)
    a = np.array([0.7, -1.3, 2.1])
    A = a[0] * X + a[1] * Y + a[2] * Z + 0.25
    rng = np.random.default_rng(1)
    h = np.array(cv.voxel_size(GRID, BBOX))
    t = rng.uniform(1, np.array(GRID) - 2, (50, 3))
    P = np.array(BBOX[:3]) + (t + 0.5) * h
    L = level.iso_level(A, P, GRID, BBOX)
    assert abs(L - np.mean(P @ a + 0.25)) < 1e-13


def test_brute_trilinear_and_dropped_points():
    rng = np.random.default_rng(2)
    A = rng.standard_normal(GRID[::-1])
    h = np.array(cv.voxel_size(GRID, BBOX))
    bmin = np.array(BBOX[:3])
    t = rng.uniform(1, np.array(GRID) - 2, (20, 3))
    P = bmin + (t + 0.5) * h
    Pout = np.concatenate([P, bmin + (np.array([[0.2, 3, 3]]) + 0.5) * h])   # dropped
    ref = []
    for p in P:
        tt = (p - bmin) / h - 0.5
        i = np.floor(tt).astype(int)
        f = tt - i
        s = 0.0
        for dz in (0, 1):
            for dy in (0, 1):
                for dx in (0, 1):
                    w = ((f[0] if dx else 1 - f[0]) * (f[1] if dy else 1 - f[1])
                         * (f[2] if dz else 1 - f[2]))
                    s += w * A[i[2] + dz, i[1] + dy, i[0] + dx]
        ref.append(s)
    assert abs(level.iso_level(A, Pout, GRID, BBOX) - np.mean(ref)) < 1e-13
    assert S.accepted_mask(Pout, GRID, BBOX).sum() == len(P)
