"""The GPU Hausdorff distance (eq. (4)) searches each row outwards from the
pixel and stops once the horizontal offset alone exceeds the best squared
distance found, on top of per-column vertical distances.  That search is
restated here step by step and checked against the oracle's brute force on
random silhouettes, so a wrong stopping rule or column sweep would show on
the CPU."""

import numpy as np

from oracle import evaluate as ev

NONE = 1 << 28


def _columns(m):
    h, w = m.shape
    col = np.full((h, w), NONE, np.int64)
    for x in range(w):
        last = -1
        for y in range(h):
            if m[y, x]:
                last = y
            col[y, x] = y - last if last >= 0 else NONE
        nxt = -1
        for y in range(h - 1, -1, -1):
            if m[y, x]:
                nxt = y
            if nxt >= 0:
                col[y, x] = min(col[y, x], nxt - y)
    return col


def _row_min(colrow, x):
    w = len(colrow)
    best = None
    for d in range(w):
        if best is not None and d * d >= best:
            break
        for xx in ((x - d,) if d == 0 else (x - d, x + d)):
            if 0 <= xx < w and colrow[xx] != NONE:
                v = d * d + int(colrow[xx]) ** 2
                best = v if best is None else min(best, v)
    return best


def _hausdorff_search(r, g):
    if not r.any() and not g.any():
        return 0.0
    if not r.any() or not g.any():
        return float("inf")
    colG, colR = _columns(g), _columns(r)
    worst = 0
    for y in range(r.shape[0]):
        for x in range(r.shape[1]):
            if r[y, x]:
                worst = max(worst, _row_min(colG[y], x))
            if g[y, x]:
                worst = max(worst, _row_min(colR[y], x))
    return float(np.sqrt(worst))


def test_row_search_equals_brute_force():
    rng = np.random.default_rng(11)
    for density in (0.02, 0.2, 0.6):
        for _ in range(4):
            r = rng.random((23, 31)) < density
            g = rng.random((23, 31)) < density * 0.5
            dr = np.where(r, 1.0, 0.0)
            dg = np.where(g, 1.0, 0.0)
            assert _hausdorff_search(r, g) == ev.hausdorff(dr, dg)
    # far-apart silhouettes: the search runs the whole row
    r = np.zeros((9, 40), bool)
    g = np.zeros((9, 40), bool)
    r[4, 0] = True
    g[0, 39] = True
    assert _hausdorff_search(r, g) == ev.hausdorff(r * 1.0, g * 1.0) == np.sqrt(39 ** 2 + 4 ** 2)
