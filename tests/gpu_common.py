"""Shared helpers of the GPU parity tests: the seeded workloads and the metrics.

The expected values always come from ``oracle/`` run on the same seeded
inputs; nothing here computes reconstruction arithmetic of its own.
"""

import functools

import numpy as np

from datagen import f32_box, frame_config, human_frame, sphere_points
from oracle import conventions as cv
from oracle import pipeline


def require_gpu():
    import pytest
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for the -m gpu tests")
    from paper_1712_03084_gb300 import build
    build.build()
    return torch


# name -> (grid_n, bbox, input generator kwargs)
CASES = {
    "sphere64": dict(kind="sphere", grid=(64, 64, 64), bbox=(-1.2, -1.2, -1.2, 1.2, 1.2, 1.2)),
    "sphere48_simple": dict(kind="sphere", grid=(48, 48, 48), bbox=(-1.2, -1.2, -1.2, 1.2, 1.2, 1.2),
                            mode=cv.SPLAT_SIMPLE),
    "human96": dict(kind="human", grid=(96, 96, 96), bbox=frame_config("human96")["bbox"], seed=11),
    "human_aniso": dict(kind="human", grid=(48, 96, 48), bbox=(-0.75, -0.05, -0.75, 0.75, 1.95, 0.75), seed=12),
    "human128": dict(kind="human", grid=(128, 128, 128), bbox=frame_config("human128")["bbox"], seed=13),
    # dense: ~3000 (point, brick) pairs per 8^3 brick, so bricks span several accumulation chunks
    "sphere32_dense": dict(kind="sphere", grid=(32, 32, 32), bbox=(-1.2, -1.2, -1.2, 1.2, 1.2, 1.2), n=60000),
}

SMALL_VIEWS = dict(depth_wh=(256, 212), fxy=182.5, rgb_wh=(480, 270), rgb_f=265.0)


@functools.lru_cache(maxsize=None)
def case_inputs(name):
    c = CASES[name]
    if c["kind"] == "sphere":
        P, N, W = sphere_points(c.get("n", 20000), 0.005, seed=0)
        return P, N, W, None
    fr = human_frame(seed=c["seed"], **SMALL_VIEWS)
    return fr["points"], fr["normals"], fr["weights"], fr["views"]


@functools.lru_cache(maxsize=None)
def oracle_result(name):
    c = CASES[name]
    P, N, W, views = case_inputs(name)
    # the oracle gets the box exactly as the kernels do (float32 coordinates)
    return pipeline.reconstruct(P, N, W, c["grid"], f32_box(c["bbox"]), mode=c.get("mode", cv.SPLAT_WEIGHTED))


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def hausdorff(a, b, chunk=4096):
    """Symmetric Hausdorff distance between two point sets (brute force, chunked)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)

    def one_way(p, q):
        worst = 0.0
        for s in range(0, len(p), chunk):
            d2 = ((p[s:s + chunk, None, :] - q[None, :, :]) ** 2).sum(-1)
            worst = max(worst, float(np.sqrt(d2.min(axis=1)).max()))
        return worst
    if len(a) == 0 or len(b) == 0:
        return 0.0 if len(a) == len(b) else float("inf")
    if len(a) * len(b) > 4e8:
        from scipy.spatial import cKDTree
        da, _ = cKDTree(b).query(a)
        db, _ = cKDTree(a).query(b)
        return float(max(da.max(), db.max()))
    return max(one_way(a, b), one_way(b, a))
