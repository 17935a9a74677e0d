"""Tile plans of the y, z and inverse-y FFT passes (8, 16 or 32 lines per CTA;
-16: the y pass with its tiles fetched by bulk asynchronous copies).

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


def _field(F, name, plan=None):
    c = G.CASES[name]
    P, N, W, _ = G.case_inputs(name)
    ctx = F.Context(c["grid"], c["bbox"], splat_mode=c.get("mode", cv.SPLAT_WEIGHTED))
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
    for plan in itertools.product(*choices):
        A, L = _field(ftr, name, plan)
        assert np.array_equal(A, ref_A), plan
        assert L == ref_L, plan


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
    plan = a.plan()
    assert rep.shape == (3, 4) and (rep[:, 1] > 0).all()       # F = 16 always fits and is timed
    for p, f in enumerate(plan):
        col = (8, 16, 32, -16).index(f)
        assert rep[p, col] > 0 and rep[p, col] == rep[p][rep[p] > 0].min()
    b = ftr.Context(c["grid"], c["bbox"])
    rep_b = b.autotune()
    assert b.plan() == plan and not rep_b.any()                   # from the cache, untimed
    # the tuned context still reconstructs the same field
    P, N, W, _ = G.case_inputs("human128")
    b.reset()
    b.splat(P, N, W)
    b.solve()
    A = b.field_A()
    a.close()
    b.close()
    ref, _ = _field(ftr, "human128", (16, 16, 16))
    assert np.array_equal(A, ref)
