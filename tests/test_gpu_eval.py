"""Rendering and the objective evaluation metrics (Sec. III-C, III-E) on the
GPU against the oracle, on the oracle's own meshes and images.

Bars: rendered depth bit-exact (coverage and depth are float64 decisions in
one fixed operation order on both sides); colours within 1 LSB (float32
barycentrics on the GPU; a multitexture pixel may move by 2 where a uv
rounding difference meets a steep texture edge, on at most 0.1% of the
pixels); silhouette counts, VRE and the Hausdorff distance exact (integer
arithmetic); CP-RMSE and each closest-point distance within 1e-6 m (every
back-projected coordinate is rounded to float32, <= 2.4e-7 m at 4 m, so a
distance moves by at most 2 sqrt(3) 2.4e-7 m); WMS3IM and its per-scale
terms within 1e-4 (float32 luma and window moments).
"""

import numpy as np
import pytest

from oracle import evaluate as oev
from oracle import render as orender
from oracle import texture as otex
from tests import gpu_common as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ftr():
    G.require_gpu()
    from paper_1712_03084_gb300 import ftr as F
    return F


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(torch.device("cuda", 0))


@pytest.fixture(scope="module")
def human(ftr):
    """The oracle's human96 mesh, its texture data and the case's views."""
    name = "human96"
    views = G.case_inputs(name)[3]
    mesh = G.oracle_result(name)["mesh"]
    verts = mesh["vertices"].astype(np.float32)
    tris = mesh["tris"].astype(np.int32)
    tex = otex.texture(verts.astype(np.float64), views, float(np.float32(0.03)))
    return {"views": views, "verts": verts, "tris": tris, "tex": tex, "grid": G.CASES[name]["grid"],
            "bbox": G.CASES[name]["bbox"]}


def _render(ftr, torch, ctx, verts, tris, K, RT, w, h, **colour):
    cam = ftr.make_camera(K, RT, w, h)
    depth = torch.zeros((h, w), dtype=torch.float32, device="cuda")
    rgb = torch.zeros((h, w, 3), dtype=torch.uint8, device="cuda") if colour else None
    ftr.ftr_render(ctx.h, _dev(torch, verts), _dev(torch, tris), cam, depth, rgb, **colour)
    return cam, depth, rgb


def test_depth_is_bit_exact_in_every_view(ftr, human):
    import torch
    ctx = ftr.Context(human["grid"], human["bbox"])
    for v in human["views"]:
        for K, RT, (h, w) in ((v["K"], v["world_to_cam"], v["depth"].shape),
                              (v["K_rgb"], v["world_to_rgb"], v["rgb"].shape[:2])):
            _, depth, _ = _render(ftr, torch, ctx, human["verts"], human["tris"], K, RT, w, h)
            ref, win = orender.rasterise(human["verts"], human["tris"], K, RT, w, h)
            got = depth.cpu().numpy()
            assert (win >= 0).sum() > 1000
            assert np.array_equal(got, ref)
    ctx.close()


def test_vertex_colour_and_multitexture(ftr, human):
    import torch
    ctx = ftr.Context(human["grid"], human["bbox"])
    views, tex = human["views"], human["tex"]
    dviews = [{"depth": _dev(torch, v["depth"]), "rgb": _dev(torch, v["rgb"]), "K": v["K"],
               "world_to_cam": v["world_to_cam"]} for v in views]
    for v in views[:2]:
        K, RT, (h, w) = v["K_rgb"], v["world_to_rgb"], v["rgb"].shape[:2]
        _, d1, c1 = _render(ftr, torch, ctx, human["verts"], human["tris"], K, RT, w, h,
                            vertex_rgb=_dev(torch, tex["rgb"]))
        rd, rc = orender.render_vertex_colour(human["verts"], human["tris"], tex["rgb"], K, RT, w, h)
        assert np.array_equal(d1.cpu().numpy(), rd)
        assert np.max(np.abs(c1.cpu().numpy().astype(int) - rc.astype(int))) <= 1
        _, d2, c2 = _render(ftr, torch, ctx, human["verts"], human["tris"], K, RT, w, h,
                            tex_weights=_dev(torch, tex["weights"].astype(np.float32)),
                            tex_uv=_dev(torch, tex["uv"].astype(np.float32)), tex_views=dviews)
        md, mc = orender.render_multitexture(human["verts"], human["tris"], tex["weights"].astype(np.float32),
                                             tex["uv"].astype(np.float32), views, K, RT, w, h)
        assert np.array_equal(d2.cpu().numpy(), md)
        diff = np.abs(c2.cpu().numpy().astype(int) - mc.astype(int)).max(axis=-1)
        assert diff.max() <= 2 and (diff > 1).mean() <= 1e-3
        assert (mc.sum(-1) > 0).sum() > 0.5 * (md > 0).sum()
    ctx.close()


def test_geometry_metrics(ftr, human):
    import torch
    ctx = ftr.Context(human["grid"], human["bbox"])
    for v in human["views"]:
        K, RT, (h, w) = v["K"], v["world_to_cam"], v["depth"].shape
        rd, _ = orender.rasterise(human["verts"], human["tris"], K, RT, w, h)
        gd = v["depth"].astype(np.float32)
        cam = ftr.make_camera(K, RT, w, h)
        d2 = torch.zeros((h, w), dtype=torch.float32, device="cuda")
        got = ftr.ftr_eval_geometry(ctx.h, cam, _dev(torch, rd), _dev(torch, gd), d2)
        vre, x, o, nr, ng = oev.vre(rd, gd)
        assert (got["xor_px"], got["or_px"], got["rendered_px"], got["sensor_px"]) == (x, o, nr, ng)
        assert got["vre"] == vre
        assert got["hausdorff_px"] == oev.hausdorff(rd, gd)
        rmse, I, J = oev.cp_rmse(K, rd, gd)
        assert (got["sensor_points"], got["rendered_points"]) == (I, J)
        assert abs(got["cp_rmse"] - rmse) <= 1e-6
        # per-pixel closest-point distances
        Xg, Xr = oev.backproject(K, gd), oev.backproject(K, rd)
        ref = np.sqrt(oev.closest_sq(Xg, Xr))
        jj, ii = np.nonzero(gd > 0)
        d = d2.cpu().numpy()
        assert np.max(np.abs(np.sqrt(d[jj, ii]) - ref)) <= 1e-6
        assert np.all(d[gd <= 0] == 0)
    ctx.close()


def test_appearance_metric(ftr, human):
    import torch
    ctx = ftr.Context(human["grid"], human["bbox"])
    views, tex = human["views"], human["tex"]
    for v in views[:2]:
        K, RT, (h, w) = v["K_rgb"], v["world_to_rgb"], v["rgb"].shape[:2]
        rd, rc = orender.render_multitexture(human["verts"], human["tris"], tex["weights"].astype(np.float32),
                                             tex["uv"].astype(np.float32), views, K, RT, w, h)
        got = ftr.ftr_eval_appearance(ctx.h, _dev(torch, rd), _dev(torch, rc), _dev(torch, v["rgb"]))
        ref, L, C, S = oev.wms3im(rd, rc, v["rgb"])
        assert 0.3 < ref < 1.0
        assert abs(got["wms3im"] - ref) <= 1e-4
        for a, b in ((got["l"], L), (got["c"], C), (got["s"], S)):
            assert np.max(np.abs(np.array(a) - np.array(b))) <= 1e-4
    ctx.close()


def test_edge_cases(ftr):
    import torch
    ctx = ftr.Context((32, 32, 32), (-1.0, -1.0, -1.0, 1.0, 1.0, 1.0))
    K = np.array([[50.0, 0, 16.0], [0, 50.0, 12.0], [0, 0, 1.0]], np.float32)
    RT = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1).astype(np.float32)
    verts = np.array([[-0.2, -0.2, 2.0], [0.3, -0.1, 2.0], [0.0, 0.3, 2.5]], np.float32)
    # no triangles; a triangle with an index out of range; a 1 x 1 image
    for tris, (w, h) in ((np.zeros((0, 3), np.int32), (32, 24)), (np.array([[0, 1, 7]], np.int32), (32, 24)),
                         (np.array([[0, 1, 2]], np.int32), (1, 1))):
        cam = ftr.make_camera(K, RT, w, h)
        depth = torch.full((h, w), -1.0, dtype=torch.float32, device="cuda")
        ftr.ftr_render(ctx.h, _dev(torch, verts), _dev(torch, tris), cam, depth, n_vertices=3)
        valid = tris[(tris >= 0).all(1) & (tris < 3).all(1)]
        ref, _ = orender.rasterise(verts, valid, K, RT, w, h)
        assert np.array_equal(depth.cpu().numpy(), ref)
    with pytest.raises(ftr.FtrError):
        ftr.ftr_render(ctx.h, _dev(torch, verts), _dev(torch, np.array([[0, 1, 2]], np.int32)),
                       ftr.make_camera(K, RT, 0, 4), torch.zeros((4, 1), device="cuda"))
    # empty silhouettes
    cam = ftr.make_camera(K, RT, 32, 24)
    zero = np.zeros((24, 32), np.float32)
    one = zero.copy()
    one[5:9, 7:12] = 2.0
    g = ftr.ftr_eval_geometry(ctx.h, cam, _dev(torch, zero), _dev(torch, one))
    assert g["hausdorff_px"] == float("inf") and g["cp_rmse"] == float("inf") and g["vre"] == 1.0
    g = ftr.ftr_eval_geometry(ctx.h, cam, _dev(torch, one), _dev(torch, zero))
    assert np.isnan(g["cp_rmse"]) and g["sensor_points"] == 0
    g = ftr.ftr_eval_geometry(ctx.h, cam, _dev(torch, zero), _dev(torch, zero))
    assert g["hausdorff_px"] == 0.0 and g["vre"] == 0.0
    img = np.random.default_rng(0).integers(0, 256, (24, 32, 3)).astype(np.uint8)
    a = ftr.ftr_eval_appearance(ctx.h, _dev(torch, zero), _dev(torch, img), _dev(torch, img))
    assert np.isnan(a["wms3im"])
    tiny = np.full((3, 3), 1.0, np.float32)
    a = ftr.ftr_eval_appearance(ctx.h, _dev(torch, tiny), _dev(torch, img[:3, :3]), _dev(torch, img[:3, :3]))
    assert np.isnan(a["wms3im"]) and np.isnan(oev.wms3im(tiny, img[:3, :3], img[:3, :3])[0])
    big = zero.copy()
    big[2:22, 3:30] = 1.5
    a = ftr.ftr_eval_appearance(ctx.h, _dev(torch, big), _dev(torch, img), _dev(torch, img))
    assert abs(a["wms3im"] - 1.0) <= 1e-5
    ctx.close()


def test_large_triangles_share_their_pixels(ftr):
    """Triangles with more than 1024 pixel centres in their box go to the
    CTA-shared pass; the depth stays bit-exact, including where they meet
    small triangles in front of them."""
    import torch
    ctx = ftr.Context((32, 32, 32), (-1.0, -1.0, -1.0, 1.0, 1.0, 1.0))
    RT = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1).astype(np.float32)
    K = np.array([[1060.0, 0, 960.0], [0, 1060.0, 540.0], [0, 0, 1.0]], np.float32)
    # a tilted quad filling the view, one mid-size triangle and a small one in front
    quad = [[-2.0, -1.2, 2.5], [2.0, -1.2, 3.5], [2.0, 1.2, 3.5], [-2.0, 1.2, 2.5]]
    mid = [[-0.3, -0.2, 2.0], [0.2, -0.25, 2.1], [0.0, 0.3, 2.05]]
    small = [[0.01, 0.01, 1.5], [0.02, 0.01, 1.5], [0.01, 0.02, 1.5]]
    verts = np.array(quad + mid + small, np.float32)
    tris = np.array([[0, 1, 2], [0, 2, 3], [4, 5, 6], [7, 8, 9]], np.int32)
    _, depth, _ = _render(ftr, torch, ctx, verts, tris, K, RT, 1920, 1080)
    ref, win = orender.rasterise(verts, tris, K, RT, 1920, 1080)
    assert (win == 0).sum() > 500000 and (win == 2).sum() > 10000 and (win == 3).sum() > 0
    assert np.array_equal(depth.cpu().numpy(), ref)
    ctx.close()


def _uv_sphere(r, centre, n_th=181, n_ph=361):
    th, ph = np.meshgrid(np.linspace(0, np.pi, n_th), np.linspace(0, 2 * np.pi, n_ph), indexing="ij")
    P = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], -1).reshape(-1, 3) * r + centre
    a, b = np.meshgrid(np.arange(n_th - 1), np.arange(n_ph - 1), indexing="ij")
    i0 = (a * n_ph + b).ravel()
    i1, i2, i3 = i0 + 1, i0 + n_ph, i0 + n_ph + 1
    tris = np.concatenate([np.stack([i0, i2, i1], 1), np.stack([i1, i2, i3], 1)]).astype(np.int32)
    return P.astype(np.float32), tris


def test_full_size_views(ftr):
    """A 130k-triangle sphere in the 512 x 424 depth and 1920 x 1080 RGB
    cameras of the human frames: depth bit-exact, geometry metrics against a
    sensor silhouette of a displaced sphere, WMS3IM at 1920 x 1080."""
    import torch
    ctx = ftr.Context((64, 64, 64), (-1.0, -1.0, -1.0, 1.0, 1.0, 1.0))
    verts, tris = _uv_sphere(0.25, np.array([0.05, -0.02, 2.6]))
    RT = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1).astype(np.float32)
    Kd = np.array([[365.0, 0, 256.0], [0, 365.0, 212.0], [0, 0, 1.0]], np.float32)
    Kc = np.array([[1060.0, 0, 960.0], [0, 1060.0, 540.0], [0, 0, 1.0]], np.float32)
    cam, depth, _ = _render(ftr, torch, ctx, verts, tris, Kd, RT, 512, 424)
    rd, _ = orender.rasterise(verts, tris, Kd, RT, 512, 424)
    assert np.array_equal(depth.cpu().numpy(), rd)
    sverts, stris = _uv_sphere(0.26, np.array([0.0, 0.0, 2.62]), 61, 121)
    gd, _ = orender.rasterise(sverts, stris, Kd, RT, 512, 424)
    got = ftr.ftr_eval_geometry(ctx.h, cam, _dev(torch, rd), _dev(torch, gd))
    vre, x, o, nr, ng = oev.vre(rd, gd)
    assert (got["xor_px"], got["or_px"]) == (x, o) and got["hausdorff_px"] == oev.hausdorff(rd, gd)
    assert abs(got["cp_rmse"] - oev.cp_rmse(Kd, rd, gd)[0]) <= 1e-6
    # colour at 1920 x 1080: vertex colours from the position
    col = np.clip(128 + 400 * (verts - verts.mean(0)), 0, 255).astype(np.uint8)
    _, dc, cc = _render(ftr, torch, ctx, verts, tris, Kc, RT, 1920, 1080, vertex_rgb=_dev(torch, col))
    rdc, rcc = orender.render_vertex_colour(verts, tris, col, Kc, RT, 1920, 1080)
    assert np.array_equal(dc.cpu().numpy(), rdc)
    assert np.max(np.abs(cc.cpu().numpy().astype(int) - rcc.astype(int))) <= 1
    sensor = np.clip(rcc.astype(int) + np.random.default_rng(1).integers(-20, 21, rcc.shape), 0, 255).astype(np.uint8)
    a = ftr.ftr_eval_appearance(ctx.h, _dev(torch, rdc), _dev(torch, rcc), _dev(torch, sensor))
    ref = oev.wms3im(rdc, rcc, sensor)
    assert abs(a["wms3im"] - ref[0]) <= 1e-4
    ctx.close()
