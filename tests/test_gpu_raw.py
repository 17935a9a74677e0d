"""Raw reconstruction on the device (Sec. III-A) against the oracle.

ftr_splat_depth turns depth maps into points, normals and confidences on the
GPU and appends them to the frame.  Bars: the confidence maps W_k within
1e-5 of the oracle's, the number of points exact, the splatted field V within 1e-5 (max abs) of the oracle's
splat of the oracle's raw points, and the indicator, level and mesh to the
end-to-end bars of the point path (A rel-L2 1e-5, |dL|/span 1e-5, vertex
Hausdorff 0.5 voxel).
"""

import numpy as np
import pytest

from datagen import f32_box
from oracle import pipeline
from oracle import raw as oraw
from oracle import splat as osplat
from tests import gpu_common as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ftr():
    G.require_gpu()
    from paper_1712_03084_gb300 import ftr as F
    return F


def _device_views(torch, views):
    dev = torch.device("cuda", 0)
    out = []
    for v in views:
        d = {"depth": torch.from_numpy(np.ascontiguousarray(v["depth"])).to(dev), "K": v["K"],
             "world_to_cam": v["world_to_cam"]}
        out.append(d)
    return out


def _oracle_raw(views):
    P, N, W, maps = [], [], [], []
    for v in views:
        p, n, w, m = oraw.raw_points(v["depth"], v["K"], v["world_to_cam"])
        P.append(p)
        N.append(n)
        W.append(w)
        maps.append(m)
    return np.concatenate(P), np.concatenate(N), np.concatenate(W), maps


def test_device_points_equal_the_oracle_points(ftr):
    """Points, normals and W written by the raw reconstruction, one by one
    against oracle.raw.raw_points on the same depth maps (Sec. III-A): same
    count and pixel order, positions within 4e-6 m (the kernel works in
    float32 on coordinates up to ~3 m, whose ulp is 2.4e-7 m: about a dozen
    roundings), unit normals within 1e-5, W within 1e-5."""
    import torch
    fr_views = G.case_inputs("human96")[3]
    dviews = _device_views(torch, fr_views)
    ctx = ftr.Context(G.CASES["human96"]["grid"], G.CASES["human96"]["bbox"])
    ctx.reset()
    ftr.ftr_splat_depth(ctx.h, dviews)
    n_in, _ = ctx.stats()
    pixels = sum(int(v["depth"].numel()) for v in dviews)
    buf = np.zeros(7 * pixels, np.float32)
    ftr.ftr_debug_buffer(ctx.h, 2, buf)
    ctx.close()
    P, N, W, _ = _oracle_raw(fr_views)
    assert n_in == len(P) > 1000
    gp = buf[:3 * pixels].reshape(pixels, 3)[:n_in]
    gn = buf[3 * pixels:6 * pixels].reshape(pixels, 3)[:n_in]
    gw = buf[6 * pixels:][:n_in]
    assert np.abs(gp - P).max() <= 4e-6
    assert np.abs(gn - N).max() <= 1e-5
    assert np.abs(gw - W).max() <= 1e-5


@pytest.mark.parametrize("name", ["human96", "human128"])
def test_depth_maps_to_field_and_mesh(ftr, name):
    import torch
    c = G.CASES[name]
    fr_views = G.case_inputs(name)[3]
    dviews = _device_views(torch, fr_views)
    confs = [torch.zeros(v["depth"].shape, dtype=torch.float32, device="cuda") for v in dviews]
    ctx = ftr.Context(c["grid"], c["bbox"])
    ctx.reset()
    ftr.ftr_splat_depth(ctx.h, dviews, conf_out=confs)
    n_in, _ = ctx.stats()
    L = ctx.solve()
    V = ctx.field_V()
    A = ctx.field_A()
    verts = ctx.mesh_numpy()["vertices"]
    ctx.close()
    P, N, W, maps = _oracle_raw(fr_views)
    assert n_in == len(P)
    for got, ref in zip(confs, maps):
        assert np.abs(got.cpu().numpy() - ref).max() <= 1e-5
    box = f32_box(c["bbox"])
    Vref = osplat.splat(P.astype(np.float32), N.astype(np.float32), W.astype(np.float32), c["grid"], box)
    assert np.abs(V - Vref).max() <= 1e-5
    ref = pipeline.reconstruct(P.astype(np.float32), N.astype(np.float32), W.astype(np.float32), c["grid"], box)
    assert G.rel_l2(A, ref["A"]) <= 1e-5
    span = float(ref["A"].max() - ref["A"].min())
    assert abs(L - ref["L"]) / span <= 1e-5
    h = max((c["bbox"][3 + a] - c["bbox"][a]) / c["grid"][a] for a in range(3))
    assert G.hausdorff(verts, ref["mesh"]["vertices"]) <= 0.5 * h


def test_edge_cases(ftr):
    """An empty view adds nothing; a lone pixel or a 2 x 2 map with one quad
    follows the triangle rule; the smallest window radius works."""
    import torch
    dev = torch.device("cuda", 0)
    K = np.array([[100.0, 0, 20.0], [0, 100.0, 15.0], [0, 0, 1.0]], np.float32)
    RT = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1).astype(np.float32)
    ctx = ftr.Context((64, 64, 64), (-1.2, -1.2, -1.2, 1.2, 1.2, 1.2))
    empty = np.zeros((30, 40), np.float32)
    lone = empty.copy()
    lone[10, 10] = 1.0
    quad = np.ones((2, 2), np.float32)
    for D, radius in [(empty, 10), (lone, 10), (quad, 0), (quad, 16)]:
        dv = {"depth": torch.from_numpy(D).to(dev), "K": K, "world_to_cam": RT}
        conf = torch.full(D.shape, -1.0, dtype=torch.float32, device=dev)
        ctx.reset()
        ftr.ftr_splat_depth(ctx.h, [dv], radius=radius, conf_out=[conf])
        n_in, _ = ctx.stats()
        p, n, w, m = oraw.raw_points(D, K, RT, radius=radius)
        assert n_in == len(p)
        assert np.abs(conf.cpu().numpy() - m).max() <= 1e-6
    with pytest.raises(ftr.FtrError):
        ftr.ftr_splat_depth(ctx.h, [{"depth": torch.from_numpy(quad).to(dev), "K": K, "world_to_cam": RT}],
                            radius=17)
    ctx.close()


def test_async_depth_path_equals_the_waiting_one(ftr):
    """ftr_splat_depth_async (device-side point count, no host wait) gives the
    same field and level as ftr_splat_depth, inside a whole-frame graph too,
    and enforces being the frame's only point source."""
    import torch
    c = G.CASES["human96"]
    dviews = _device_views(torch, G.case_inputs("human96")[3])
    ctx = ftr.Context(c["grid"], c["bbox"])
    ctx.reset()
    ftr.ftr_splat_depth(ctx.h, dviews)
    n_sync, _ = ctx.stats()
    L0 = ctx.solve()
    A0 = ctx.field_A()
    ctx.reset()
    ftr.ftr_splat_depth(ctx.h, dviews, wait=False)
    n_async, _ = ctx.stats()
    L1 = ctx.solve()
    A1 = ctx.field_A()
    assert n_async == n_sync and L1 == L0 and np.array_equal(A1, A0)
    with pytest.raises(ftr.FtrError):
        ftr.ftr_splat(ctx.h, np.zeros((1, 3), np.float32), np.zeros((1, 3), np.float32))
    for _ in range(2):               # graph capture, then replay
        ctx.reset()
        ftr.ftr_splat_depth(ctx.h, dviews, wait=False)
        ftr.ftr_frame_launch(ctx.h, [], 0.02)
        m = ftr.ftr_frame_finish(ctx.h)
    assert np.array_equal(ctx.field_A(), A0)
    ctx.reset()
    ftr.ftr_splat(ctx.h, np.zeros((1, 3), np.float32), np.zeros((1, 3), np.float32))
    with pytest.raises(ftr.FtrError):
        ftr.ftr_splat_depth(ctx.h, dviews, wait=False)
    ctx.close()
