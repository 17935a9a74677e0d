"""GPU path vs the FP64 oracle, stage by stage, through the C ABI.

Bars (FP32 kernels against the float64 oracle on the same float32 inputs):
  V            max |V_gpu - V_oracle| <= 1e-5 (|V| <= sqrt(1.5))
  A            relative L2 <= 1e-5
  L            |L_gpu - L_oracle| / (max A - min A) <= 1e-5
  MC on the oracle's A (rounded to float32) and L: cube classes, vertex and
               triangle counts and the triangle index lists bit-exact; vertex
               positions within 1e-6 of the float64 lerp, normals within 1e-4
  end to end   vertex Hausdorff between the GPU and oracle meshes <= 0.5 voxel
The grids cover several tiles and bricks, radix-3 lengths (48, 96), the
paper's 2^r x 2^(r+1) x 2^r anisotropy and the simple splat variant.
"""

import numpy as np
import pytest

from oracle import conventions as cv
from oracle import mc as omc
from tests import gpu_common as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ftr():
    G.require_gpu()
    from paper_1712_03084_gb300 import ftr as F
    return F


def _run(F, name, **kw):
    c = G.CASES[name]
    P, N, W, _ = G.case_inputs(name)
    ctx = F.Context(c["grid"], c["bbox"], splat_mode=c.get("mode", cv.SPLAT_WEIGHTED), **kw)
    ctx.reset()
    ctx.splat(P, N, W)
    L = ctx.solve()
    return ctx, L


@pytest.mark.parametrize("name", list(G.CASES))
def test_splat_field_V(ftr, name):
    ctx, _ = _run(ftr, name)
    V = ctx.field_V()
    ref = G.oracle_result(name)["V"]
    assert np.max(np.abs(V - ref)) <= 1e-5
    ctx.close()


@pytest.mark.parametrize("name", list(G.CASES))
def test_indicator_and_level(ftr, name):
    ctx, L = _run(ftr, name)
    A = ctx.field_A()
    r = G.oracle_result(name)
    assert G.rel_l2(A, r["A"]) <= 1e-5
    span = float(r["A"].max() - r["A"].min())
    assert abs(L - r["L"]) / span <= 1e-5
    ctx.close()


@pytest.mark.parametrize("name", list(G.CASES))
def test_both_transform_paths_match_the_oracle(ftr, name):
    """The plane-fused transforms (forward x+y and inverse y+x per z-plane in
    one thread-block cluster) and the five axis passes both meet the A and L
    bars against the oracle, and agree with each other to rounding."""
    c = G.CASES[name]
    P, N, W, _ = G.case_inputs(name)
    r = G.oracle_result(name)
    span = float(r["A"].max() - r["A"].min())
    got = {}
    for path in (1, 0):
        ctx = ftr.Context(c["grid"], c["bbox"], splat_mode=c.get("mode", cv.SPLAT_WEIGHTED))
        ctx.set_transform_path(path)                  # path 1 is built for every parity grid
        ctx.reset()
        ctx.splat(P, N, W)
        L = ctx.solve()
        A = ctx.field_A()
        ctx.close()
        assert G.rel_l2(A, r["A"]) <= 1e-5, path
        assert abs(L - r["L"]) / span <= 1e-5, path
        got[path] = A
    assert G.rel_l2(got[1], got[0]) <= 2e-6


@pytest.mark.parametrize("name", ["sphere64", "human96", "human128"])
def test_persistent_y_z_pass_equals_the_five_passes(ftr, name):
    """Transform path 2 (the y pass and the z pass in one persistent kernel,
    the intermediate handed over through an L2 ring of k_x planes) runs the
    per-line arithmetic of the five passes with 16-line tiles: A and L agree
    with them to rounding (the two kernels are compiled separately, so the
    last bits may differ) and with the oracle within its bars, also over two
    frames in a row (the ring and the counters are reused); both frames of
    path 2 are bit-identical (the handover order does not change a value)."""
    c = G.CASES[name]
    P, N, W, _ = G.case_inputs(name)
    res = {}
    for path in (0, 2):
        ctx = ftr.Context(c["grid"], c["bbox"])
        ctx.set_transform_path(path)
        ctx.set_plan((16, 16, 16))
        out = []
        for _ in range(2):
            ctx.reset()
            ctx.splat(P, N, W)
            out.append((ctx.solve(), ctx.field_A()))
        ctx.close()
        res[path] = out
    r = G.oracle_result(name)
    span = float(r["A"].max() - r["A"].min())
    for (L0, A0), (L2, A2) in zip(res[0], res[2]):
        assert G.rel_l2(A2, A0) <= 1e-6 and abs(L2 - L0) / span <= 1e-7
        assert G.rel_l2(A2, r["A"]) <= 1e-5 and abs(L2 - r["L"]) / span <= 1e-5
    assert res[2][0][0] == res[2][1][0] and np.array_equal(res[2][0][1], res[2][1][1])


@pytest.mark.parametrize("name", ["sphere64", "human96", "human_aniso"])
def test_marching_cubes_bit_exact_on_oracle_field(ftr, name):
    c = G.CASES[name]
    r = G.oracle_result(name)
    A32 = r["A"].astype(np.float32)
    L = r["L"]
    ref = omc.marching_cubes(A32.astype(np.float64), L, c["grid"], G.f32_box(c["bbox"]))
    ctx = ftr.Context(c["grid"], c["bbox"])
    ctx.set_indicator(A32, L)
    assert np.array_equal(ctx.cube_classes(), ref["classes"].astype(np.uint8))
    m = ctx.mesh_numpy()
    assert len(m["vertices"]) == len(ref["vertices"])
    assert len(m["tris"]) == len(ref["tris"])
    assert np.array_equal(m["tris"], ref["tris"].astype(np.int32))
    assert np.max(np.abs(m["vertices"] - ref["vertices"])) <= 1e-6 * max(1.0, np.abs(ref["vertices"]).max())
    assert np.max(np.abs(m["normals"] - ref["normals"])) <= 1e-4
    ctx.close()


@pytest.mark.parametrize("name", ["sphere64", "human96", "human128"])
def test_end_to_end_mesh_hausdorff(ftr, name):
    c = G.CASES[name]
    ctx, _ = _run(ftr, name)
    m = ctx.mesh_numpy()
    ref = G.oracle_result(name)["mesh"]
    h = min(cv.voxel_size(c["grid"], c["bbox"]))
    assert abs(len(m["vertices"]) - len(ref["vertices"])) <= 0.01 * len(ref["vertices"]) + 10
    assert G.hausdorff(m["vertices"], ref["vertices"]) <= 0.5 * h
    ctx.close()


def test_deterministic_and_host_device_inputs_agree(ftr):
    import torch
    name = "human96"
    c = G.CASES[name]
    P, N, W, _ = G.case_inputs(name)
    outs = []
    for dev in (False, True, True):
        ctx = ftr.Context(c["grid"], c["bbox"])
        if dev:
            ctx.splat(torch.from_numpy(P).cuda(), torch.from_numpy(N).cuda(), torch.from_numpy(W).cuda())
        else:
            ctx.splat(P, N, W)
        L = ctx.solve()
        outs.append((L, ctx.field_A(), ctx.mesh_numpy()))
        ctx.close()
    for L, A, m in outs[1:]:
        assert L == outs[0][0]
        assert np.array_equal(A, outs[0][1])
        assert np.array_equal(m["tris"], outs[0][2]["tris"])
        assert np.array_equal(m["vertices"], outs[0][2]["vertices"])


def test_splat_is_additive_over_calls(ftr):
    """One call per camera equals one call with all points (exact fixed-point sums)."""
    name = "human96"
    c = G.CASES[name]
    P, N, W, _ = G.case_inputs(name)
    ctx = ftr.Context(c["grid"], c["bbox"])
    ctx.splat(P, N, W)
    L1 = ctx.solve()
    V1 = ctx.field_V()
    ctx.reset()
    cuts = np.linspace(0, len(P), 5).astype(int)
    for a, b in zip(cuts[:-1], cuts[1:]):
        ctx.splat(P[a:b].copy(), N[a:b].copy(), W[a:b].copy())
    L2 = ctx.solve()
    assert np.array_equal(V1, ctx.field_V())
    assert L1 == L2
    ctx.close()


def test_edge_cases(ftr):
    grid = (32, 32, 32)
    box = (-1.0, -1.0, -1.0, 1.0, 1.0, 1.0)
    ctx = ftr.Context(grid, box)
    # empty frame
    L = ctx.solve()
    assert L == 0.0
    assert np.all(ctx.field_A() == 0)
    m = ctx.mesh_numpy()
    assert len(m["tris"]) == 0
    # every point outside the accepted region: dropped and counted
    P = np.array([[0.99, 0.0, 0.0], [-0.97, 0.1, 0.1], [np.nan, 0, 0]], np.float32)
    N = np.tile(np.array([[1.0, 0, 0]], np.float32), (3, 1))
    ctx.reset()
    ctx.splat(P, N, None)
    assert ctx.stats() == (3, 3)
    assert ctx.solve() == 0.0
    # a single point: V has its 4^3 stencil and nothing else
    ctx.reset()
    ctx.splat(np.array([[0.1, -0.2, 0.3]], np.float32), np.array([[0, 0, 1.0]], np.float32), None)
    ctx.solve()
    V = ctx.field_V()
    assert np.count_nonzero(np.any(V != 0, axis=0)) == 64
    ctx.close()
    # invalid calls are rejected and leave the context usable
    ctx = ftr.Context(grid, box)
    with pytest.raises(ftr.FtrError):
        ftr.ftr_extract_mesh(ctx.h)
    ftr.ftr_splat(ctx.h, np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32), None)   # n = 0 is fine
    assert ctx.solve() == 0.0
    ctx.close()


def test_texture_matches_oracle_on_the_same_mesh(ftr):
    """Sec. III-C per-vertex weights, UVs and blended colour of the oracle's
    mesh, textured on the GPU (ftr_texture_vertices) and by the oracle."""
    import torch
    from oracle import texture as otex
    name = "human96"
    c = G.CASES[name]
    P, N, W, views = G.case_inputs(name)
    verts = G.oracle_result(name)["mesh"]["vertices"].astype(np.float32)
    nv, k = len(verts), len(views)
    dev = torch.device("cuda", 0)
    dviews = [{key: (torch.from_numpy(np.ascontiguousarray(v[key])).to(dev) if key in ("depth", "conf", "rgb")
                     else v[key]) for key in v} for v in views]
    w = torch.zeros((nv, k), dtype=torch.float32, device=dev)
    uv = torch.zeros((nv, k, 2), dtype=torch.float32, device=dev)
    rgb = torch.zeros((nv, 3), dtype=torch.uint8, device=dev)
    tx = torch.zeros((nv,), dtype=torch.uint8, device=dev)
    ctx = ftr.Context(c["grid"], c["bbox"])
    tol = float(np.float32(0.03))
    ftr.ftr_texture_vertices(ctx.h, dviews, tol, torch.from_numpy(verts).to(dev), w, uv, rgb, tx)
    tex = {"weights": w.cpu().numpy(), "uv": uv.cpu().numpy(), "rgb": rgb.cpu().numpy(), "textured": tx.cpu().numpy()}
    ref = otex.texture(verts.astype(np.float64), views, tol)
    assert np.array_equal(tex["weights"] > 0, ref["weights"] > 0)
    assert np.array_equal(tex["weights"], ref["weights"].astype(np.float32))
    vis = ref["weights"] > 0
    assert vis.mean() > 0.3
    assert np.max(np.abs(tex["uv"][vis] - ref["uv"][vis])) <= 1e-3
    assert np.all(tex["uv"][~vis] == -1)
    assert np.array_equal(tex["textured"], ref["textured"])
    assert np.max(np.abs(tex["rgb"].astype(int) - ref["rgb"].astype(int))) <= 1
    # ftr_texture on the context's own mesh = ftr_texture_vertices on those vertices
    r = G.oracle_result(name)
    ctx.set_indicator(r["A"].astype(np.float32), r["L"])
    m = ctx.mesh_numpy()
    own = ctx.texture_numpy(views, tol, len(m["vertices"]))
    n2 = len(m["vertices"])
    w2 = torch.zeros((n2, k), dtype=torch.float32, device=dev)
    rgb2 = torch.zeros((n2, 3), dtype=torch.uint8, device=dev)
    ftr.ftr_texture_vertices(ctx.h, dviews, tol, torch.from_numpy(m["vertices"]).to(dev), w2, None, rgb2, None)
    assert np.array_equal(own["weights"], w2.cpu().numpy()) and np.array_equal(own["rgb"], rgb2.cpu().numpy())
    ctx.close()


def test_texture_matches_oracle_on_full_size_views(ftr):
    """The texture stage at the benchmark frame's image sizes (four 512 x 424
    depth maps, four 1920 x 1080 RGB views, Sec. III-C): the oracle's 128^3
    mesh of that frame textured by ftr_texture_vertices and by the oracle.
    Weights bit-equal, UVs within 1e-3 px, colours within 1 LSB."""
    import torch
    from datagen import f32_box, frame_config, human_frame
    from oracle import pipeline
    from oracle import texture as otex
    cfg = frame_config("human128")
    fr = human_frame(seed=1, K=cfg["K"], ring=cfg["ring"], height=cfg["height"])
    views = fr["views"]
    assert views[0]["depth"].shape == (424, 512) and views[0]["rgb"].shape == (1080, 1920, 3)
    ref_mesh = pipeline.reconstruct(fr["points"], fr["normals"], fr["weights"], cfg["grid_n"],
                                    f32_box(cfg["bbox"]))["mesh"]
    verts = ref_mesh["vertices"].astype(np.float32)
    nv, k = len(verts), len(views)
    dev = torch.device("cuda", 0)
    dviews = [{key: (torch.from_numpy(np.ascontiguousarray(v[key])).to(dev) if key in ("depth", "conf", "rgb")
                     else v[key]) for key in v} for v in views]
    w = torch.zeros((nv, k), dtype=torch.float32, device=dev)
    uv = torch.zeros((nv, k, 2), dtype=torch.float32, device=dev)
    rgb = torch.zeros((nv, 3), dtype=torch.uint8, device=dev)
    tx = torch.zeros((nv,), dtype=torch.uint8, device=dev)
    ctx = ftr.Context(cfg["grid_n"], cfg["bbox"])
    tol = float(np.float32(0.03))
    ftr.ftr_texture_vertices(ctx.h, dviews, tol, torch.from_numpy(verts).to(dev), w, uv, rgb, tx)
    ctx.close()
    ref = otex.texture(verts.astype(np.float64), views, tol)
    assert np.array_equal(w.cpu().numpy(), ref["weights"].astype(np.float32))
    vis = ref["weights"] > 0
    assert vis.mean() > 0.3
    assert np.max(np.abs(uv.cpu().numpy()[vis] - ref["uv"][vis])) <= 1e-3
    assert np.all(uv.cpu().numpy()[~vis] == -1)
    assert np.array_equal(tx.cpu().numpy(), ref["textured"])
    assert np.max(np.abs(rgb.cpu().numpy().astype(int) - ref["rgb"].astype(int))) <= 1


def test_async_frame_equals_sync_frame(ftr):
    """Queued frame (extract/texture async, one wait) = the waiting calls."""
    import torch
    name = "human96"
    c = G.CASES[name]
    P, N, W, views = G.case_inputs(name)
    tol = float(np.float32(0.03))
    ctx, _ = _run(ftr, name)
    m_sync = ctx.mesh_numpy()
    t_sync = ctx.texture_numpy(views, tol, len(m_sync["vertices"]))
    dviews = []
    for v in views:
        d = dict(v)
        for key in ("depth", "conf", "rgb"):
            d[key] = torch.from_numpy(v[key]).cuda()
        dviews.append(d)
    cap = ftr.ftr_mesh_capacity(ctx.h)
    K = len(views)
    w = torch.zeros((cap, K), dtype=torch.float32, device="cuda")
    uv = torch.zeros((cap, K, 2), dtype=torch.float32, device="cuda")
    rgb = torch.zeros((cap, 3), dtype=torch.uint8, device="cuda")
    tx = torch.zeros((cap,), dtype=torch.uint8, device="cuda")
    for _ in range(2):
        ctx.reset()
        ctx.splat(P, N, W)
        ctx.solve(want_level=False)
        ftr.ftr_extract_mesh_async(ctx.h)
        ftr.ftr_texture_async(ctx.h, dviews, tol, w, uv, rgb, tx, cap)
        m = ftr.ftr_frame_finish(ctx.h)
        nv = m.n_vertices
        assert nv == len(m_sync["vertices"]) and m.n_tris == len(m_sync["tris"])
        v = np.zeros((nv, 3), np.float32)
        t = np.zeros((m.n_tris, 3), np.int32)
        ftr.ftr_mesh_copy(ctx.h, v, None, t)
        assert np.array_equal(v, m_sync["vertices"]) and np.array_equal(t, m_sync["tris"])
        assert np.array_equal(w[:nv].cpu().numpy(), t_sync["weights"])
        assert np.array_equal(rgb[:nv].cpu().numpy(), t_sync["rgb"])
        assert np.array_equal(tx[:nv].cpu().numpy(), t_sync["textured"])
    ctx.close()


def test_async_mesh_grows_past_its_first_capacity(ftr):
    """A field with far more surface than the first buffers: finish grows and redoes the mesh."""
    grid = (64, 64, 64)
    box = (0.0, 0.0, 0.0, 1.0, 1.0, 1.0)
    A = np.random.default_rng(8).standard_normal((64, 64, 64)).astype(np.float32)
    ref_ctx = ftr.Context(grid, box)
    ref_ctx.set_indicator(A, 0.0)
    ref = ref_ctx.mesh_numpy()
    ref_ctx.close()
    ctx = ftr.Context(grid, box)
    ctx.set_indicator(A, 0.0)
    ftr.ftr_extract_mesh_async(ctx.h)
    assert ftr.ftr_mesh_capacity(ctx.h) < len(ref["vertices"])
    m = ftr.ftr_frame_finish(ctx.h)
    assert m.n_vertices == len(ref["vertices"]) and m.n_tris == len(ref["tris"])
    v = np.zeros((m.n_vertices, 3), np.float32)
    t = np.zeros((m.n_tris, 3), np.int32)
    ftr.ftr_mesh_copy(ctx.h, v, None, t)
    assert np.array_equal(v, ref["vertices"]) and np.array_equal(t, ref["tris"])
    ctx.close()


def test_graph_frame_equals_separate_calls(ftr):
    """ftr_frame_launch (one CUDA graph per frame) = solve + async extract + async texture,
    also when the point count changes between replays."""
    import torch
    name = "human96"
    c = G.CASES[name]
    P, N, W, views = G.case_inputs(name)
    tol = float(np.float32(0.03))
    dviews = []
    for v in views:
        d = dict(v)
        for key in ("depth", "conf", "rgb"):
            d[key] = torch.from_numpy(v[key]).cuda()
        dviews.append(d)
    K = len(views)
    cap = 200000
    outs = [torch.zeros((cap, K), dtype=torch.float32, device="cuda"),
            torch.zeros((cap, K, 2), dtype=torch.float32, device="cuda"),
            torch.zeros((cap, 3), dtype=torch.uint8, device="cuda"),
            torch.zeros((cap,), dtype=torch.uint8, device="cuda")]
    g = ftr.Context(c["grid"], c["bbox"])
    for sub in (len(P), len(P) // 2, len(P)):
        ref = ftr.Context(c["grid"], c["bbox"])
        ref.splat(P[:sub].copy(), N[:sub].copy(), W[:sub].copy())
        L = ref.solve()
        m_ref = ref.mesh_numpy()
        t_ref = ref.texture_numpy(views, tol, len(m_ref["vertices"]))
        ref.close()
        g.reset()
        g.splat(P[:sub].copy(), N[:sub].copy(), W[:sub].copy())
        ftr.ftr_frame_launch(g.h, dviews, tol, *outs, out_capacity=cap)
        m = ftr.ftr_frame_finish(g.h)
        nv = m.n_vertices
        assert nv == len(m_ref["vertices"]) and m.n_tris == len(m_ref["tris"])
        v = np.zeros((nv, 3), np.float32)
        t = np.zeros((m.n_tris, 3), np.int32)
        ftr.ftr_mesh_copy(g.h, v, None, t)
        assert np.array_equal(v, m_ref["vertices"]) and np.array_equal(t, m_ref["tris"])
        assert np.array_equal(outs[0][:nv].cpu().numpy(), t_ref["weights"])
        assert np.array_equal(outs[2][:nv].cpu().numpy(), t_ref["rgb"])
    g.close()


def test_graph_frame_follows_new_view_buffers(ftr):
    """Frames whose views live in other device buffers (other images, other
    calibrations) give the texture data of those views: the graph's texture
    node takes the new view set (or the frame is captured again)."""
    import torch
    name = "human96"
    c = G.CASES[name]
    P, N, W, views = G.case_inputs(name)
    other = G.case_inputs("human128")[3]            # another rig and other images, same sizes
    tol = float(np.float32(0.03))

    def dev(vs, invert):
        out = []
        for v in vs:
            d = dict(v)
            for key in ("depth", "conf", "rgb"):
                a = v[key]
                if key == "rgb" and invert:
                    a = (255 - a).astype(np.uint8)
                d[key] = torch.from_numpy(np.ascontiguousarray(a)).cuda()
            out.append(d)
        return out
    sets = [dev(views, False), dev(views, True), dev(other, False)]
    K = len(views)
    cap = 200000
    outs = [torch.zeros((cap, K), dtype=torch.float32, device="cuda"),
            torch.zeros((cap, K, 2), dtype=torch.float32, device="cuda"),
            torch.zeros((cap, 3), dtype=torch.uint8, device="cuda"),
            torch.zeros((cap,), dtype=torch.uint8, device="cuda")]
    g = ftr.Context(c["grid"], c["bbox"])
    for j in (0, 1, 2, 0, 2, 1):
        g.reset()
        g.splat(P, N, W)
        ftr.ftr_frame_launch(g.h, sets[j], tol, *outs, out_capacity=cap)
        m = ftr.ftr_frame_finish(g.h)
        nv = m.n_vertices
        ref = g.texture_numpy(sets[j], tol, nv)
        assert np.array_equal(outs[0][:nv].cpu().numpy(), ref["weights"])
        assert np.array_equal(outs[2][:nv].cpu().numpy(), ref["rgb"])
    g.close()


@pytest.mark.parametrize("name", ["sphere64", "human_aniso"])
def test_inside_mask_is_the_binarised_volume(ftr, name):
    """The exported binarised volume (Sec. IV's input) is exactly A >= L of
    the solved field and level, and matches the oracle's classification."""
    ctx, L = _run(ftr, name)
    A = ctx.field_A()
    m = ctx.inside_mask()
    ctx.close()
    assert np.array_equal(m, A.astype(np.float64) >= L)
    r = G.oracle_result(name)
    agree = np.mean(m == (r["A"] >= r["L"]))
    assert agree > 0.9999


def test_point_sets_in_one_launch_equal_separate_calls(ftr):
    """ftr_splat_sets (every camera's points ingested by one launch) stores
    exactly what one ftr_splat call per camera stores: the same V, A, L and
    the same counts, with device sets and with host (staged) sets."""
    import torch
    name = "human96"
    c = G.CASES[name]
    P, N, W, _ = G.case_inputs(name)
    dev = torch.device("cuda", 0)
    Pd, Nd, Wd = (torch.from_numpy(x).to(dev) for x in (P, N, W))
    cuts = [0, 5000, 5001, 17000, len(P)]
    sets = [(Pd[a:b], Nd[a:b], Wd[a:b]) for a, b in zip(cuts[:-1], cuts[1:])]
    sets.append((Pd[:0], Nd[:0], None))                    # an empty set is allowed
    host_sets = [(P[a:b], N[a:b], W[a:b]) for a, b in zip(cuts[:-1], cuts[1:])]
    res = []
    for mode in ("one launch", "host sets", "separate calls"):
        ctx = ftr.Context(c["grid"], c["bbox"])
        ctx.reset()
        l0 = ctx.launch_count()
        if mode == "one launch":
            ctx.splat_sets(sets)
            assert ctx.launch_count() - l0 == 1
        elif mode == "host sets":
            ctx.splat_sets(host_sets)
            assert ctx.launch_count() - l0 == 1
        else:
            for p, n, w in sets:
                ctx.splat(p, n, w)
        L = ctx.solve()
        res.append((ctx.field_V(), ctx.field_A(), L, ctx.stats()))
        ctx.close()
    for V2, A2, L2, s2 in res[1:]:
        V1, A1, L1, s1 = res[0]
        assert np.array_equal(V1, V2) and np.array_equal(A1, A2) and L1 == L2 and s1 == s2
