"""Batched frames and the continuous-batching serving loop (GPU).

Each frame's result must be the same alone and in the mix: every slot owns
its context, the splat is exact integer arithmetic and every kernel is
deterministic, so meshes are compared bit for bit.
"""

import numpy as np
import pytest

from datagen import human_frame
from tests import gpu_common as G

pytestmark = pytest.mark.gpu

BOX = (-1.0, -0.05, -1.0, 1.0, 1.95, 1.0)


@pytest.fixture(scope="module")
def rt():
    G.require_gpu()
    from paper_1712_03084_gb300 import serve
    return serve


def _frames(seed, n, K=3):
    out = []
    for i in range(n):
        fr = human_frame(seed=seed + i, K=K, **G.SMALL_VIEWS)
        out.append(fr)
    return out


def _same(a, b):
    return a.keys() == b.keys() and all(np.array_equal(a[k], b[k]) for k in a)


def test_batch_matches_sequential_and_alone(rt):
    """Vertices, triangles and every texture output of each frame are
    bit-identical whether the batch runs all at once, one frame after another,
    or the frame runs alone on a fresh slot."""
    grids = [(64, 64, 64), (96, 96, 96), (64, 128, 64), (96, 96, 96)]
    frs = _frames(50, 4)
    fins = [rt.FrameInput.from_frame(f) for f in frs]
    boxes = [BOX] * 4
    _, par = rt.run_batch(fins, grids, boxes, results=True)
    _, seq = rt.run_batch(fins, grids, boxes, sequential=True, results=True)
    for a, b in zip(par, seq):
        assert len(a["vertices"]) > 1000 and _same(a, b)
    for i in range(4):
        s = rt.Slot(grids[i], BOX, fins[i], fins[i].n_points)
        s.submit(fins[i])
        s.finish()
        alone = s.results()
        s.close()
        assert _same(alone, par[i]), i


def test_server_mix_equals_alone_and_reports_latency(rt):
    specs = [((64, 64, 64), 3, 60), ((96, 96, 96), 4, 70), ((64, 64, 64), 3, 80)]
    sessions = []
    for sid, (grid, K, seed) in enumerate(specs):
        fins = [rt.FrameInput.from_frame(f) for f in _frames(seed, 2, K)]
        sessions.append(rt.Session(sid, grid, BOX, fins, rate_hz=60.0))
    srv = rt.Server(hbm_budget_bytes=64 << 30)
    for s in sessions:
        assert srv.admit(s)
    keep = {(0, 0), (1, 1), (2, 0)}
    stats = srv.run(duration_s=0.4, seed=3, keep_meshes=keep)
    srv.close()
    assert stats["frames"] > 10 and stats["p99_ms"] >= stats["p50_ms"] > 0
    for (sid, k), (v, t) in stats["meshes"].items():
        sess = sessions[sid]
        alone = rt.Slot(sess.grid_n, BOX, sess.frames[0], max(f.n_points for f in sess.frames))
        alone.submit(sess.frames[k % len(sess.frames)])
        alone.finish()
        va, ta = alone.mesh()
        alone.close()
        assert np.array_equal(v, va) and np.array_equal(t, ta)
    assert len(stats["meshes"]) >= 2


def test_estimate_bounds_the_slot_after_its_frames(rt):
    """The admission estimate (no allocation) is at least what a slot holds
    after running every frame of its session, and not far above it."""
    fins = [rt.FrameInput.from_frame(f) for f in _frames(95, 2, K=4)]
    sess = rt.Session(0, (96, 96, 96), BOX, fins)
    est = rt.slot_estimate_bytes(sess)
    s = rt.Slot(sess.grid_n, BOX, fins[0], max(f.n_points for f in fins))
    for f in fins:
        s.submit(f)
        s.finish()
    real = s.device_bytes()
    s.close()
    assert real <= est <= 3 * real


def test_admission_respects_the_hbm_budget(rt):
    fins = [rt.FrameInput.from_frame(f) for f in _frames(90, 1)]
    probe = rt.Slot((96, 96, 96), BOX, fins[0], fins[0].n_points)
    one = probe.device_bytes()
    probe.close()
    srv = rt.Server(hbm_budget_bytes=int(one * 1.5))
    a = rt.Session(0, (96, 96, 96), BOX, fins)
    b = rt.Session(1, (96, 96, 96), BOX, fins)
    assert srv.admit(a) and not srv.admit(b)
    assert srv.rejected == [1] and srv.used <= srv.budget
    srv.close()


def test_rgbd_sessions_match_the_device_raw_path_alone(rt):
    """Sessions fed as RGB-D images (points, normals and W maps computed on
    the device without a host wait) give, in the mix, the meshes of a lone
    context running the waiting raw-reconstruction call on the same images."""
    import torch
    from paper_1712_03084_gb300 import ftr
    specs = [((64, 64, 64), 3, 110), ((96, 96, 96), 4, 120)]
    sessions = []
    for sid, (grid, K, seed) in enumerate(specs):
        frs = _frames(seed, 2, K)
        fins = [rt.FrameInput.from_frame(f, rgbd=True) for f in frs]
        sessions.append(rt.Session(sid, grid, BOX, fins, rate_hz=60.0))
    srv = rt.Server(hbm_budget_bytes=64 << 30)
    for s in sessions:
        assert srv.admit(s)
    keep = {(0, 0), (1, 1)}
    stats = srv.run(duration_s=0.4, seed=5, keep_meshes=keep)
    srv.close()
    assert stats["frames"] > 10
    for (sid, k), (v, t) in stats["meshes"].items():
        sess = sessions[sid]
        fin = sess.frames[k % len(sess.frames)]
        views = [{"depth": x["depth"].cuda(), "K": x["K"], "world_to_cam": x["world_to_cam"]} for x in fin.views]
        ctx = ftr.Context(sess.grid_n, BOX)
        ctx.reset()
        ftr.ftr_splat_depth(ctx.h, views)
        ctx.solve()
        m = ctx.mesh_numpy()
        ctx.close()
        assert np.array_equal(v, m["vertices"]) and np.array_equal(t, m["tris"])
    assert len(stats["meshes"]) == 2


def test_fetch_async_reads_back_the_frame(rt):
    """Slot.fetch_async (ftr_mesh_copy_async + texture copies, no host wait)
    lands the same mesh and texture data as the waiting reads, also while the
    other slot of a two-slot pipeline is busy."""
    fins = [rt.FrameInput.from_frame(f) for f in _frames(130, 2)]
    slots = [rt.Slot((96, 96, 96), BOX, fins[0], max(f.n_points for f in fins)) for _ in range(2)]
    hosts = [s.host_buffers() for s in slots]
    for s, f in zip(slots, fins):
        s.submit(f)
    for s, h, f in zip(slots, hosts, fins):
        nv, nt = s.finish()
        s.fetch_async(h)
        s.submit(f)                       # the next frame queued behind the read-back
        s.fetched.synchronize()
        assert nv > 1000 and h["vertices"][:nv].abs().sum() > 0
    for s, h in zip(slots, hosts):
        s.finish()
        v, t = s.mesh()
        s.fetch_async(h)
        s.fetched.synchronize()
        nv, nt = len(v), len(t)
        assert np.array_equal(h["vertices"][:nv].numpy(), v) and np.array_equal(h["tris"][:nt].numpy(), t)
        assert np.array_equal(h["weights"][:nv].numpy(), s.out_w[:nv].cpu().numpy())
        assert np.array_equal(h["rgb"][:nv].numpy(), s.out_rgb[:nv].cpu().numpy())
        s.close()
