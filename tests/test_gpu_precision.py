"""Split-precision tensor-core FFT passes against the FP64 oracle.

With FTR_PREC_BF16X3 / FTR_PREC_FP16X3 every small DFT of the transforms is a
tensor-core product of 16-bit hi/lo operand parts accumulated in fp32
(x D ~ x_lo D_hi + x_hi D_lo + x_hi D_hi).  Per product the neglected part is
x_lo D_lo plus the rounding of the lo parts, at most about 3 u^2 of |x| |D|
with u = 2^-9 (bf16) or 2^-11 (fp16) — 1.1e-5 and 7e-7.  The indicator goes
through twelve such stages (two per axis, forward and inverse), whose errors
add roughly in quadrature, plus the fp32 twiddles and filter.  Bars on A
(relative L2 against the oracle) and on L (|dL| / (max A - min A)):
  BF16X3   2e-4   (about 4x the sqrt(12) * 1.1e-5 estimate)
  FP16X3   1e-5   (the fp32 path's own bar)
and the mesh within half a voxel (Hausdorff) of the oracle's.
"""

import numpy as np
import pytest

from oracle import conventions as cv
from tests import gpu_common as G

pytestmark = pytest.mark.gpu

BAR = {1: 2e-4, 2: 1e-5}
NAMES = {1: "bf16x3", 2: "fp16x3"}


@pytest.fixture(scope="module")
def ftr():
    G.require_gpu()
    from paper_1712_03084_gb300 import ftr as F
    return F


def _solve(F, name, prec):
    c = G.CASES[name]
    P, N, W, _ = G.case_inputs(name)
    ctx = F.Context(c["grid"], c["bbox"], splat_mode=c.get("mode", cv.SPLAT_WEIGHTED), precision=prec)
    ctx.reset()
    ctx.splat(P, N, W)
    L = ctx.solve()
    return ctx, L


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("name", ["sphere64", "human128"])
def test_indicator_and_level(ftr, name, prec):
    ctx, L = _solve(ftr, name, prec)
    A = ctx.field_A()
    ctx.close()
    r = G.oracle_result(name)
    err = G.rel_l2(A, r["A"])
    span = float(r["A"].max() - r["A"].min())
    dl = abs(L - r["L"]) / span
    print(f"{name} {NAMES[prec]}: A rel-L2 {err:.3e}, |dL|/span {dl:.3e}")
    assert err <= BAR[prec]
    assert dl <= BAR[prec]


@pytest.mark.parametrize("prec", [1, 2])
def test_mesh_against_oracle(ftr, prec):
    name = "human128"
    ctx, _ = _solve(ftr, name, prec)
    m = ctx.mesh_numpy()
    ctx.close()
    r = G.oracle_result(name)
    c = G.CASES[name]
    h = max((c["bbox"][3 + a] - c["bbox"][a]) / c["grid"][a] for a in range(3))
    d = G.hausdorff(m["vertices"], r["mesh"]["vertices"])
    print(f"{name} {NAMES[prec]}: vertex Hausdorff {d / h:.3e} voxels")
    assert d <= 0.5 * h


@pytest.mark.parametrize("prec", [1, 2])
def test_graph_frame_matches_separate_calls(ftr, prec):
    """The whole-frame graph (captured on first use) replays the split-precision
    passes exactly like the separate calls."""
    import torch
    name = "human128"
    c = G.CASES[name]
    P, N, W, _ = G.case_inputs(name)
    dev = torch.device("cuda", 0)
    Pd = torch.from_numpy(np.ascontiguousarray(P)).to(dev)
    Nd = torch.from_numpy(np.ascontiguousarray(N)).to(dev)
    Wd = torch.from_numpy(np.ascontiguousarray(W)).to(dev)
    ctx = ftr.Context(c["grid"], c["bbox"], precision=prec)
    got = []
    for _ in range(2):
        ctx.reset()
        ftr.ftr_splat(ctx.h, Pd, Nd, Wd)
        ftr.ftr_frame_launch(ctx.h, [], 0.02)
        m = ftr.ftr_frame_finish(ctx.h)
        v = np.zeros((m.n_vertices, 3), np.float32)
        t = np.zeros((m.n_tris, 3), np.int32)
        ftr.ftr_mesh_copy(ctx.h, v, None, t)
        got.append((v, t))
    ctx.reset()
    ctx.splat(P, N, W)
    ctx.solve()
    ref = ctx.mesh_numpy()
    ctx.close()
    for v, t in got:
        assert np.array_equal(v, ref["vertices"])
        assert np.array_equal(t, ref["tris"])


@pytest.mark.parametrize("prec,which", [(1, 0), (0, 1)])
def test_a_timed_out_wait_is_reported_and_the_context_recovers(ftr, prec, which):
    """A bounded device wait that gives up sets a flag that the next waiting
    call turns into FTR_ETIMEOUT.  The flag is raised from the host here (no
    GPU wait is made to run out): ftr_solve reports FTR_ETIMEOUT once, clears
    the flag, and the next frame on the same context is right again."""
    name = "sphere64"
    c = G.CASES[name]
    P, N, W, _ = G.case_inputs(name)
    ctx = ftr.Context(c["grid"], c["bbox"], precision=prec)
    ctx.reset()
    ctx.splat(P, N, W)
    L0 = ctx.solve()
    ftr.ftr_debug_raise_wait_flag(ctx.h, which)
    ctx.reset()
    ctx.splat(P, N, W)
    with pytest.raises(ftr.FtrError) as e:
        ctx.solve()
    assert e.value.code == ftr.FTR_ETIMEOUT
    ctx.reset()
    ctx.splat(P, N, W)
    assert ctx.solve() == L0
    if prec == 0:
        with pytest.raises(ftr.FtrError):
            ftr.ftr_debug_raise_wait_flag(ctx.h, 0)       # an FP32 context has no tensor-core flag
    ctx.close()
