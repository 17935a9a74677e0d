"""Split-precision transform passes with a 384-point axis, against the oracle.

The 384-point plan (384 = 24 x 16) has its own tile shapes in the
tensor-core passes (the z pass takes 8 lines per CTA there, the others 16)
and the longest small DFTs (R = 24).  Each grid puts 384 on x, on y or on z
in turn, the other axes at 64 nodes (every axis of a split-precision
context must be 64, 128, 256 or 384 long), so that the FP64 oracle finishes
in seconds (Sec. III-B).

Bars as in test_gpu_precision.py, from the split-operand arithmetic: A
relative L2 and |dL| / span(A) within 2e-4 (bf16 parts) and 1e-5 (fp16
parts, scaled per line); the mesh within half a voxel (Hausdorff).
"""

import functools

import numpy as np
import pytest

from datagen import f32_box, sphere_points
from oracle import pipeline
from tests import gpu_common as G

pytestmark = pytest.mark.gpu

BOX = (-1.2, -1.2, -1.2, 1.2, 1.2, 1.2)
GRIDS = {"x384": (384, 64, 64), "y384": (64, 384, 64), "z384": (64, 64, 384)}
BAR = {1: 2e-4, 2: 1e-5}


@pytest.fixture(scope="module")
def ftr():
    G.require_gpu()
    from paper_1712_03084_gb300 import ftr as F
    return F


@functools.lru_cache(maxsize=None)
def _inputs():
    return sphere_points(20000, 0.005, seed=3)


@functools.lru_cache(maxsize=None)
def _oracle(name):
    P, N, W = _inputs()
    return pipeline.reconstruct(P, N, W, GRIDS[name], f32_box(BOX))


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("name", list(GRIDS))
def test_split_precision_long_axis_against_the_oracle(ftr, name, prec):
    grid = GRIDS[name]
    P, N, W = _inputs()
    ctx = ftr.Context(grid, BOX, precision=prec)
    ctx.reset()
    ctx.splat(P, N, W)
    L = ctx.solve()
    A = ctx.field_A()
    verts = ctx.mesh_numpy()["vertices"]
    ctx.close()
    r = _oracle(name)
    err = G.rel_l2(A, r["A"])
    span = float(r["A"].max() - r["A"].min())
    dl = abs(L - r["L"]) / span
    print(f"{name} precision {prec}: A rel-L2 {err:.3e}, |dL|/span {dl:.3e}")
    assert err <= BAR[prec]
    assert dl <= BAR[prec]
    h = max((BOX[3 + a] - BOX[a]) / grid[a] for a in range(3))
    assert len(verts) > 1000
    assert G.hausdorff(verts, r["mesh"]["vertices"]) <= 0.5 * h
