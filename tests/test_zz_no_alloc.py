"""The allocation-free level entry point agrees with the regular path.

``ftr_iso_level_noalloc`` serves callers that cannot allocate device memory
where they need the level (a latency-bound per-frame loop, or a host
framework that owns every allocation).  It keeps its partial sums in a static
device array, so this test calls it twice in a row through the C ABI on the
indicator and points of a real frame and checks both results against the
level ``ftr_solve`` returns for the same frame, with the tolerance the other
level tests use (|dL| / span(A) <= 1e-5).
"""

import numpy as np
import pytest

from tests import gpu_common as G

pytestmark = pytest.mark.gpu


def test_noalloc_level_matches_solve_twice():
    torch = G.require_gpu()
    from paper_1712_03084_gb300 import ftr
    name = "human96"
    c = G.CASES[name]
    P, N, W, _ = G.case_inputs(name)
    ctx = ftr.Context(c["grid"], c["bbox"])
    ctx.splat(P, N, W)
    L_ref = ctx.solve()
    A = ctx.field_A()
    ctx.close()
    span = float(A.max() - A.min())
    A_dev = torch.from_numpy(A).cuda()
    P_dev = torch.from_numpy(P).cuda()
    for _ in range(2):                      # the shared scratch keeps the previous call's contents
        L = ftr.ftr_iso_level_noalloc(A_dev, c["grid"], c["bbox"], P_dev)
        assert abs(L - L_ref) / span <= 1e-5
    # a device output buffer works too
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    ftr.ftr_iso_level_noalloc(A_dev, c["grid"], c["bbox"], P_dev, level_out=out)
    torch.cuda.synchronize()
    assert abs(float(out.item()) - L_ref) / span <= 1e-5
    # a different, smaller point set right after still gives its own level
    half = P_dev[: len(P) // 2].contiguous()
    L_half = ftr.ftr_iso_level_noalloc(A_dev, c["grid"], c["bbox"], half)
    assert np.isfinite(L_half) and abs(L_half - L_ref) / span < 0.1


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = G.require_gpu()
    from paper_1712_03084_gb300 import ftr
    A_dev = torch.zeros((32, 32, 32), dtype=torch.float32, device="cuda")
    P_dev = torch.zeros((1, 3), dtype=torch.float32, device="cuda")
    # the size check runs before any GPU work, so the short buffer is never read
    with pytest.raises(ftr.FtrError):
        ftr.ftr_iso_level_noalloc(A_dev, (32, 32, 32), (0, 0, 0, 1, 1, 1), P_dev, n=4 * 1024 * 1024 + 1)
