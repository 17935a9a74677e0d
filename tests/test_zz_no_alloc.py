"""The allocation-free level entry point against the oracle's level.

``ftr_iso_level_noalloc`` serves callers that cannot allocate device memory
where they need the level (a latency-bound per-frame loop, where cudaMalloc
and cudaFree may synchronise the device, or a host framework that owns every
allocation).  It keeps its partial sums in a static device array, so this
test calls it twice in a row through the C ABI on the indicator and points
of a real frame and checks both results against ``oracle.level.iso_level``
on the same float32 A and points (|dL| / span(A) <= 1e-5, the bar of the
other level tests), then against the regular path's level, then on half of
the points right after the full set (the scratch keeps the previous call's
partial sums, which must not leak into the next result).
"""

import ctypes

import numpy as np
import pytest

from datagen import f32_box
from oracle import level as olevel
from tests import gpu_common as G

pytestmark = pytest.mark.gpu


def test_noalloc_level_matches_the_oracle_twice():
    torch = G.require_gpu()
    from paper_1712_03084_gb300 import ftr
    name = "human96"
    c = G.CASES[name]
    P, N, W, _ = G.case_inputs(name)
    ctx = ftr.Context(c["grid"], c["bbox"])
    ctx.splat(P, N, W)
    L_solve = ctx.solve()
    A = ctx.field_A()
    ctx.close()
    box = f32_box(c["bbox"])
    span = float(A.max() - A.min())
    L_or = olevel.iso_level(A.astype(np.float64), P, c["grid"], box)
    L_or_half = olevel.iso_level(A.astype(np.float64), P[: len(P) // 2], c["grid"], box)
    A_dev = torch.from_numpy(A).cuda()
    P_dev = torch.from_numpy(P).cuda()
    for _ in range(2):                      # the shared scratch keeps the previous call's contents
        L = ftr.ftr_iso_level_noalloc(A_dev, c["grid"], c["bbox"], P_dev)
        assert abs(L - L_or) / span <= 1e-5
        assert abs(L - L_solve) / span <= 1e-5
    # a device output buffer works too
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    ftr.ftr_iso_level_noalloc(A_dev, c["grid"], c["bbox"], P_dev, level_out=out)
    torch.cuda.synchronize()
    assert abs(float(out.item()) - L_or) / span <= 1e-5
    # half of the points right after the full set: its own level, nothing left over
    half = P_dev[: len(P) // 2].contiguous()
    for _ in range(2):
        L_half = ftr.ftr_iso_level_noalloc(A_dev, c["grid"], c["bbox"], half)
        assert abs(L_half - L_or_half) / span <= 1e-5
    assert abs(L_or_half - L_or) / span > 1e-4          # the two sets really differ
    # no points: L = 0 (no accepted sample)
    assert ftr.ftr_iso_level_noalloc(A_dev, c["grid"], c["bbox"], P_dev, n=0) == 0.0


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = G.require_gpu()
    from paper_1712_03084_gb300 import ftr
    A_dev = torch.zeros((32, 32, 32), dtype=torch.float32, device="cuda")
    P_dev = torch.zeros((1, 3), dtype=torch.float32, device="cuda")
    out = np.zeros(1, np.float64)
    g = (ctypes.c_int * 3)(32, 32, 32)
    b = (ctypes.c_float * 6)(0, 0, 0, 1, 1, 1)
    # called below the binding, whose own checks would stop n > rows first: the
    # library's size check runs before any GPU work, so the short buffer is never read
    code = ftr.load().ftr_iso_level_noalloc(A_dev.data_ptr(), g, b, P_dev.data_ptr(), 4 * 1024 * 1024 + 1,
                                            out.ctypes.data, None)
    assert code == -1                       # FTR_EINVAL
    with pytest.raises(ValueError):
        ftr.ftr_iso_level_noalloc(A_dev, (32, 32, 32), (0, 0, 0, 1, 1, 1), P_dev, n=2)
