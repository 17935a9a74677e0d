"""The marching cubes compare float32 A with the level L rounded up to
float32 instead of promoting every A to float64: A >= L (float64) holds
exactly when A >= roundup32(L).  Checked exhaustively around random levels
(every float32 within a few ulps of L) and on random fields."""

import numpy as np


def _roundup32(L):
    f = np.float32(L)
    if np.float64(f) < L:
        f = np.nextafter(f, np.float32(np.inf))
    return f


def test_float32_threshold_equals_float64_compare():
    rng = np.random.default_rng(8)
    for L in np.concatenate([rng.standard_normal(2000) * 10.0, [0.0, -0.0, 1e-30, -1e-30, 3.0, 0.1]]):
        L = np.float64(L)
        Lf = _roundup32(L)
        c = np.float32(L)
        near = [c]
        for _ in range(4):
            near.append(np.nextafter(near[-1], np.float32(np.inf)))
        lo = [c]
        for _ in range(4):
            lo.append(np.nextafter(lo[-1], np.float32(-np.inf)))
        A = np.array(near + lo + list(rng.standard_normal(50).astype(np.float32) * 10), np.float32)
        assert np.array_equal(A >= Lf, A.astype(np.float64) >= L)
