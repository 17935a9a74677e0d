"""Pins for the oracle splat, eq. (1)(2) of Sec. III-B, no GPU needed."""

import json
import os

import numpy as np

from oracle import conventions as cv
from oracle import splat as S

GRID = (12, 10, 14)
BBOX = (-1.0, -0.5, -0.7, 1.4, 1.5, 1.1)


def _golden():
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")) as f:
        return json.load(f)


def test_constants_match_paper():
    g = _golden()
    assert cv.SIGMA2_RATIO2 == g["sigma2_sq_over_sigma1_sq"]["value"]
    assert cv.STENCIL == g["splat_support_nodes_per_axis"]["value"]
    h = cv.voxel_size(GRID, BBOX)
    s1, s2 = cv.sigmas(GRID, BBOX)
    diag = np.sqrt(sum(x * x for x in h))
    assert np.isclose(s1, g["sigma1_over_voxel_diagonal"]["value"] * diag)
    assert np.isclose(s2 * s2, 1.5 * s1 * s1)


def test_single_point_closed_form():
    """One point: V(q) = (s2/s1) exp(-r^2 (1/s1^2 - 1/s2^2)) N on its 4^3 nodes, 0 elsewhere."""
    X = np.array([[0.13, 0.41, 0.27]])
    N = np.array([[0.3, -0.5, 0.8]])
    s1, s2 = cv.sigmas(GRID, BBOX)
    for w in (0.3, 1.7):
        V = S.splat_weighted(X, N, np.array([w]), GRID, BBOX)
        nzv = np.argwhere(np.any(V != 0, axis=0))
        assert len(nzv) == 64
        t = S.node_coords(X, GRID, BBOX)[0]
        lo = np.floor(t).astype(int) - 1
        for z, y, x in nzv:
            q = np.array([x, y, z])
            assert np.all(q >= lo) and np.all(q <= lo + 3)
            r2 = np.sum((X[0] - S.node_position(q, GRID, BBOX)) ** 2)
            ref = (s2 / s1) * np.exp(-r2 * (1 / s1 ** 2 - 1 / s2 ** 2)) * N[0]
            assert np.allclose(V[:, z, y, x], ref, rtol=1e-13, atol=1e-15)


def test_stencil_brute_force():
    """All-node loop with the stencil written as -2 <= t - q < 2 (independent form)."""
    rng = np.random.default_rng(5)
    n = np.array(GRID)
    h = np.array(cv.voxel_size(GRID, BBOX))
    bmin = np.array(BBOX[:3])
    # points inside the accepted region plus a few that must be dropped
    tt = rng.uniform(1.0, n - 2.0, size=(25, 3))
    X = bmin + (tt + 0.5) * h
    X = np.concatenate([X, bmin + (np.array([[0.5, 3, 3], [3, 3, n[2] - 1.5]]) + 0.5) * h])
    N = rng.standard_normal((len(X), 3))
    W = rng.uniform(0.1, 1.0, len(X))
    s1, s2 = cv.sigmas(GRID, BBOX)
    V, U, d = S.splat_weighted(X, N, W, GRID, BBOX, return_ud=True)
    Ub = np.zeros_like(U)
    db = np.zeros_like(d)
    for i in range(len(X)):
        t = (X[i] - bmin) / h - 0.5
        if not (np.all(t >= 1) and np.all(t < n - 2)):
            continue
        for z in range(GRID[2]):
            for y in range(GRID[1]):
                for x in range(GRID[0]):
                    q = np.array([x, y, z])
                    off = t - q
                    if np.all(off >= -2) and np.all(off < 2):
                        p = bmin + (q + 0.5) * h
                        r2 = np.sum((X[i] - p) ** 2)
                        Ub[:, z, y, x] += np.exp(-r2 / s1 ** 2) / s1 * W[i] * N[i]
                        db[z, y, x] += np.exp(-r2 / s2 ** 2) / s2 * W[i]
    assert np.allclose(U, Ub, rtol=1e-12, atol=1e-14)
    assert np.allclose(d, db, rtol=1e-12, atol=1e-14)
    # |V| <= sqrt(1.5) max |N| (g1/g2 <= s2/s1 pointwise)
    assert np.max(np.linalg.norm(V, axis=0)) <= np.sqrt(1.5) * np.max(np.linalg.norm(N, axis=1)) + 1e-12


def test_acceptance_rule():
    """Accepted iff 1 <= t < n-2 per axis (binary-exact box, h = 1/4)."""
    n = np.array(GRID)
    exact_box = (0.0, 0.0, 0.0, 3.0, 2.5, 3.5)
    t = np.array([[1.0, 1.0, 1.0], [0.999, 2, 2], [n[0] - 2.0, 2, 2], [n[0] - 2.0 - 1e-6, 2, 2]])
    X = (t + 0.5) * 0.25
    assert S.accepted_mask(X, GRID, exact_box).tolist() == [True, False, False, True]


def test_simple_mode_counts():
    rng = np.random.default_rng(9)
    n = np.array(GRID)
    h = np.array(cv.voxel_size(GRID, BBOX))
    bmin = np.array(BBOX[:3])
    q = np.array([4, 5, 6])
    X = bmin + (q + 0.5 + rng.uniform(-0.49, 0.49, (7, 3))) * h
    N = rng.standard_normal((7, 3))
    V = S.splat_simple(X, N, GRID, BBOX)
    assert np.allclose(V[:, q[2], q[1], q[0]], N.mean(axis=0), rtol=1e-14)
    assert np.count_nonzero(np.any(V != 0, axis=0)) == 1
    # rounding half up: t = q + 1/2 goes to q + 1 (binary-exact box, h = 1/4)
    exact_box = (0.0, 0.0, 0.0, 3.0, 2.5, 3.5)
    X2 = (np.array([[4.5, 5.0, 6.0]]) + 0.5) * 0.25
    V2 = S.splat_simple(X2, np.array([[1.0, 0, 0]]), GRID, exact_box)
    assert V2[0, 6, 5, 5] == 1.0
