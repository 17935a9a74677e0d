"""Tile plans of the y, z and inverse-y FFT passes (8, 16 or 32 lines per CTA;
-16: the y or z pass with its tiles fetched by bulk asynchronous copies).

Every plan runs the same per-line arithmetic, so the indicator must be
bit-identical whatever the plan; the autotuner must pick a plan that fits
the grid and reuse it, untimed, for the next context of the same grid.
"""

import itertools

import numpy as np
import pytest

from oracle import conventions as cv
from tests import gpu_common as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ftr():
    G.require_gpu()
    from paper_1712_03084_gb300 import ftr as F
    return F


def _field(F, name, plan=None, path=None):
    c = G.CASES[name]
    P, N, W, _ = G.case_inputs(name)
    ctx = F.Context(c["grid"], c["bbox"], splat_mode=c.get("mode", cv.SPLAT_WEIGHTED))
    if path is not None:
        ctx.set_transform_path(path)
    if plan is not None:
        ctx.set_plan(plan)
    ctx.reset()
    ctx.splat(P, N, W)
    L = ctx.solve()
    A = ctx.field_A()
    ctx.close()
    return A, L


@pytest.mark.parametrize("name", ["human96", "human_aniso"])
def test_every_plan_is_bit_identical(ftr, name):
    c = G.CASES[name]
    ref_A, ref_L = _field(ftr, name, (16, 16, 16))
    nx, ny, nz = c["grid"]
    choices = [[f for f in (8, 16, 32) if (ny if p == 1 else nz) % f == 0] for p in range(3)]
    if nz % 16 == 0 and ny <= 256:
        choices[0].append(-16)          # the y pass with bulk-copied tiles
    if ny % 16 == 0:
        choices[1].append(-16)          # the z pass with bulk-copied tiles
    for plan in itertools.product(*choices):
        A, L = _field(ftr, name, plan)
        assert np.array_equal(A, ref_A), plan
        assert L == ref_L, plan


@pytest.mark.parametrize("name", ["human96", "human_aniso"])
def test_every_z_plan_is_bit_identical_on_the_fused_path(ftr, name):
    """The same for the z pass of the plane-fused transform path."""
    c = G.CASES[name]
    P, N, W, _ = G.case_inputs(name)
    ny = c["grid"][1]
    ref = None
    for fz in [f for f in (8, 16, 32) if ny % f == 0]:
        ctx = ftr.Context(c["grid"], c["bbox"])
        ctx.set_transform_path(1)
        ctx.set_plan((16, fz, 16))
        ctx.reset()
        ctx.splat(P, N, W)
        L = ctx.solve()
        A = ctx.field_A()
        ctx.close()
        if ref is None:
            ref = (A, L)
        assert np.array_equal(A, ref[0]) and L == ref[1], fz


def test_transform_path_is_refused_where_not_built(ftr):
    ctx = ftr.Context((64, 96, 64), (-1, -1, -1, 1, 1, 1))     # no plane kernels for 64 x 96, n_y != n_z
    assert ctx.transform_path() == 0
    for path in (1, 2, 3):
        with pytest.raises(ftr.FtrError):
            ctx.set_transform_path(path)
    ctx.close()


def test_y_z_ring_exists_only_while_its_path_is_in_use(ftr):
    """Path 2's ring (about 40 MB of k_x planes, all of them on small grids)
    and its counters are allocated when the path is set and freed when
    another is; ftr_device_bytes counts them meanwhile."""
    for grid in ((128, 128, 128), (256, 256, 256)):
        ctx = ftr.Context(grid, (-1, -1, -1, 1, 1, 1))
        b0 = ftr.ftr_device_bytes(ctx.h)
        ctx.set_transform_path(2)
        nkx = grid[0] // 2 + 1
        planes = min(nkx, max(4, (40 << 20) // (2 * 8 * grid[1] * grid[2])))
        assert ftr.ftr_device_bytes(ctx.h) - b0 == planes * 2 * grid[1] * grid[2] * 8 + (1 + 2 * nkx) * 4
        ctx.set_transform_path(1)
        assert ftr.ftr_device_bytes(ctx.h) == b0
        ctx.set_transform_path(2)
        ctx.set_transform_path(0)
        assert ftr.ftr_device_bytes(ctx.h) == b0
        ctx.close()


def test_plan_rejects_tiles_that_do_not_divide_the_grid(ftr):
    c = G.CASES["human_aniso"]          # 48 x 96 x 48: 32 does not divide n_z
    ctx = ftr.Context(c["grid"], c["bbox"])
    with pytest.raises(ftr.FtrError):
        ctx.set_plan((32, 16, 16))
    with pytest.raises(ftr.FtrError):
        ctx.set_plan((16, 12, 16))
    ctx.close()


def test_autotune_picks_a_fitting_plan_and_caches_it(ftr):
    c = G.CASES["human128"]
    a = ftr.Context(c["grid"], c["bbox"])
    rep = a.autotune()
    full = a.tune_report
    path = a.transform_path()
    assert full[12] > 0 and full[13] > 0 and full[15] > 0         # all three chains timed
    chains = {0: full[12], 1: full[13], 2: full[15]}
    assert path == int(full[14]) == min(chains, key=chains.get)
    plan = a.plan()
    assert rep.shape == (3, 4) and (rep[:, 1] > 0).all()       # F = 16 always fits and is timed
    for p, f in enumerate(plan):
        if p == 1 and path == 1:
            continue                      # the fused path's z pass has its own tile height
        col = (8, 16, 32, -16).index(f)
        assert rep[p, col] > 0 and rep[p, col] == rep[p][rep[p] > 0].min()
    b = ftr.Context(c["grid"], c["bbox"])
    rep_b = b.autotune()
    assert b.plan() == plan and not rep_b.any()                   # from the cache, untimed
    assert b.transform_path() == path
    # the tuned context still reconstructs the same field
    P, N, W, _ = G.case_inputs("human128")
    b.reset()
    b.splat(P, N, W)
    b.solve()
    A = b.field_A()
    a.close()
    b.close()
    ref, _ = _field(ftr, "human128", (16, 16, 16), path)
    assert np.array_equal(A, ref)


def test_autotune_before_the_first_frame_on_reused_memory(ftr):
    """A context timed by ftr_autotune before it has splatted anything (its
    brick table never written by a frame) runs every transform kernel on its
    initial state; on memory another context has just used and released
    this must neither read outside its buffers nor change the results."""
    c = G.CASES["human96"]
    P, N, W, _ = G.case_inputs("human96")
    ref, _ = _field(ftr, "human96")          # leaves its memory to the allocator
    ctx = ftr.Context(c["grid"], c["bbox"])
    ctx.autotune()
    plan, path = ctx.plan(), ctx.transform_path()
    ctx.reset()
    ctx.splat(P, N, W)
    L = ctx.solve()
    A = ctx.field_A()
    ctx.close()
    ref_p, ref_pL = _field(ftr, "human96", plan, path)
    assert np.array_equal(A, ref_p) and L == ref_pL
    assert G.rel_l2(A, ref) <= 2e-6


def _mesh(F, name, mc_plan=None):
    c = G.CASES[name]
    P, N, W, _ = G.case_inputs(name)
    ctx = F.Context(c["grid"], c["bbox"])
    if mc_plan is not None:
        ctx.set_mc_plan(mc_plan)
    ctx.reset()
    ctx.splat(P, N, W)
    ctx.solve()
    m = ctx.mesh_numpy()
    ctx.close()
    return m


@pytest.mark.parametrize("name", ["human96", "human_aniso"])
def test_every_marching_cubes_plan_gives_the_same_mesh(ftr, name):
    """Count/emit tiles of 128, 256 or 512 threads and 1-16 triangle CTAs per
    SM: node records, vertex ids and triangles follow node order, so the mesh
    is bit-identical whatever the block sizes."""
    ref = _mesh(ftr, name, (256, 4))
    assert len(ref["vertices"]) > 1000
    for plan in itertools.product((128, 256, 512), (1, 2, 8, 16)):
        m = _mesh(ftr, name, plan)
        for k in ("vertices", "normals", "tris"):
            assert np.array_equal(m[k], ref[k]), (plan, k)


def test_autotune_picks_a_marching_cubes_plan_on_a_meshed_frame(ftr):
    """The autotuner times the marching-cubes block sizes on the last meshed
    frame, keeps a valid choice, and the next context of the grid takes it
    from the cache; the mesh after tuning equals the untuned one.  (A grid
    that no other test tunes, so that the timing runs here.)"""
    name = "human_aniso"
    c = G.CASES[name]
    P, N, W, _ = G.case_inputs(name)
    ref = _mesh(ftr, name)
    ctx = ftr.Context(c["grid"], c["bbox"])
    ctx.reset()
    ctx.splat(P, N, W)
    ctx.solve()
    ctx.mesh_numpy()
    ctx.autotune()
    tile, per_sm = ctx.mc_plan()
    assert tile in (128, 256, 512) and per_sm in (2, 4, 8)
    ctx.reset()
    ctx.splat(P, N, W)
    ctx.solve()
    m = ctx.mesh_numpy()
    ctx.close()
    for k in ("vertices", "normals", "tris"):
        assert np.array_equal(m[k], ref[k]), k
    ctx2 = ftr.Context(c["grid"], c["bbox"])
    ctx2.autotune()                       # cached: no frame needed
    assert ctx2.mc_plan() == (tile, per_sm)
    ctx2.close()
