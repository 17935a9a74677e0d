"""Iso-level L (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. III-B: L is the average of A at the input sample locations X_k(u).
Reading: the unweighted mean over all accepted points of the trilinear
interpolation of A between the cell-centred nodes, with the cell index
clamped to the grid.  Accepted points have 1 <= t < n-2, so no clamping
happens for them.
"""

import numpy as np

from . import splat as osplat


def trilinear(A, points, grid_n, bbox):
    """Trilinear A at each point (float64); A is indexed [z, y, x]."""
    A = np.asarray(A, dtype=np.float64)
    n = np.array(grid_n)
    t = osplat.node_coords(points, grid_n, bbox)
    i0 = np.clip(np.floor(t).astype(np.int64), 0, n - 2)
    f = np.clip(t - i0, 0.0, 1.0)
    out = np.zeros(len(t))
    for dz in (0, 1):
        wz = f[:, 2] if dz else 1.0 - f[:, 2]
        for dy in (0, 1):
            wy = f[:, 1] if dy else 1.0 - f[:, 1]
            for dx in (0, 1):
                wx = f[:, 0] if dx else 1.0 - f[:, 0]
                out += wx * wy * wz * A[i0[:, 2] + dz, i0[:, 1] + dy, i0[:, 0] + dx]
    return out


def iso_level(A, points, grid_n, bbox):
    """L = mean over accepted points of trilinear A (Sec. III-B)."""
    ok = osplat.accepted_mask(points, grid_n, bbox)
    pts = np.asarray(points, dtype=np.float64)[ok]
    if len(pts) == 0:
        return 0.0
    return float(np.mean(trilinear(A, pts, grid_n, bbox)))
