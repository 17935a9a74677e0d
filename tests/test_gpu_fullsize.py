"""Full-size parity: the benchmark's 256^3 human frame and the same frame on
the 384^3 grid (the split-precision study's and the serving sessions'
largest grid), through the same whole-frame CUDA-graph call the benchmark
times, against the FP64 oracle run on the whole frame; and the splat of the
384^3 frame against the oracle's splat.

Bars as in the small-grid parity tests: A relative L2 <= 1e-5, |dL| / (max A
- min A) <= 1e-5, vertex Hausdorff <= 0.5 voxel, max |V_gpu - V_oracle| <=
1e-5.  The oracle gets the box exactly as the kernels do (float32 corners).
"""

import numpy as np
import pytest

from datagen import f32_box, frame_config, human_frame
from oracle import pipeline
from oracle import splat as osplat
from tests import gpu_common as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ftr():
    G.require_gpu()
    from paper_1712_03084_gb300 import ftr as F
    return F


@pytest.mark.parametrize("name", ["human256", "human384"])
def test_bench_frame_graph_path(ftr, name):
    import torch
    cfg = frame_config(name)
    grid, box = cfg["grid_n"], cfg["bbox"]
    fr = human_frame(seed=1, K=cfg["K"], ring=cfg["ring"], height=cfg["height"])
    dev = torch.device("cuda", 0)
    P = torch.from_numpy(fr["points"]).to(dev)
    N = torch.from_numpy(fr["normals"]).to(dev)
    W = torch.from_numpy(fr["weights"]).to(dev)
    ctx = ftr.Context(grid, box)
    for _ in range(2):        # first call captures the graph, second replays it
        ctx.reset()
        for (s, n) in fr["per_camera"]:
            ctx.splat(P[s:s + n], N[s:s + n], W[s:s + n])
        ftr.ftr_frame_launch(ctx.h, [], 0.02)
        m = ftr.ftr_frame_finish(ctx.h)
    v = np.zeros((m.n_vertices, 3), np.float32)
    t = np.zeros((m.n_tris, 3), np.int32)
    ftr.ftr_mesh_copy(ctx.h, v, None, t)
    A = ctx.field_A()
    L = ctx.solve()
    ctx.close()
    ref = pipeline.reconstruct(fr["points"], fr["normals"], fr["weights"], grid, f32_box(box))
    assert G.rel_l2(A, ref["A"]) <= 1e-5
    span = float(ref["A"].max() - ref["A"].min())
    assert abs(L - ref["L"]) / span <= 1e-5
    h = max((box[3 + a] - box[a]) / grid[a] for a in range(3))
    assert G.hausdorff(v, ref["mesh"]["vertices"]) <= 0.5 * h
    assert len(t) > 0 and t.min() >= 0 and t.max() < len(v)


def test_splat_human384(ftr):
    cfg = frame_config("human384")
    grid, box = cfg["grid_n"], cfg["bbox"]
    fr = human_frame(seed=1, K=cfg["K"], ring=cfg["ring"], height=cfg["height"])
    ctx = ftr.Context(grid, box)
    ctx.reset()
    ctx.splat(fr["points"], fr["normals"], fr["weights"])
    ctx.solve(want_level=False)
    V = ctx.field_V()
    ctx.close()
    ref = osplat.splat(fr["points"], fr["normals"], fr["weights"], grid, f32_box(box))
    assert np.max(np.abs(V - ref)) <= 1e-5
