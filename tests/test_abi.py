"""The C-ABI library loads, exports every declared entry point, and its
host-generated marching-cubes table equals the oracle's (no GPU needed)."""

import os
import re

import numpy as np
import pytest

from oracle import mc_table

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1712_03084_gb300 import build, ftr
    build.build()
    return ftr.load()


def _declared():
    with open(os.path.join(ROOT, "include", "ftr.h")) as f:
        txt = f.read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ftr_[a-z_A-Z0-9]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(lib):
    from paper_1712_03084_gb300 import ftr
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(ftr.EXPORTED) == names


def test_library_table_matches_oracle_table(lib):
    from paper_1712_03084_gb300 import ftr
    ntri, tris = ftr.ftr_mc_table()
    ont, otr = mc_table.table()
    assert np.array_equal(ntri, ont)
    assert otr.shape[1] <= ftr.MAX_TRIS_PER_CASE
    for c in range(256):
        assert np.array_equal(tris[c, :ntri[c]], otr[c, :ont[c]]), c
        assert np.all(tris[c, ntri[c]:] == -1)


def test_create_rejects_bad_grids_without_gpu(lib):
    from paper_1712_03084_gb300 import ftr
    for grid, box in [((100, 64, 64), (0, 0, 0, 1, 1, 1)), ((64, 64, 64), (0, 0, 0, 0, 1, 1)),
                      ((64, 64, 16), (0, 0, 0, 1, 1, 1))]:
        with pytest.raises(ftr.FtrError):
            ftr.ftr_create(grid, box)


def test_create_rejects_split_precision_on_unsupported_grids_without_gpu(lib):
    """The tensor-core variants need every axis in {64, 128, 256, 384}; other
    grids and unknown precision codes are rejected before any device call."""
    from paper_1712_03084_gb300 import ftr
    for grid, prec in [((96, 96, 96), ftr.FTR_PREC_BF16X3), ((64, 64, 48), ftr.FTR_PREC_FP16X3),
                       ((512, 512, 512), ftr.FTR_PREC_BF16X3), ((64, 64, 64), 3), ((64, 64, 64), -1)]:
        p = ftr.ftr_default_params()
        p.precision = prec
        with pytest.raises(ftr.FtrError):
            ftr.ftr_create(grid, (0, 0, 0, 1, 1, 1), p)


def test_product_path_does_not_touch_the_oracle():
    pkg = os.path.join(ROOT, "paper_1712_03084_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                with open(os.path.join(dirpath, f)) as fh:
                    src = fh.read()
                assert "oracle" not in re.sub(r"#.*|//.*", "", src).replace("the oracle", ""), f


def test_estimate_bytes_needs_no_device(lib):
    """ftr_estimate_bytes is host arithmetic: the grid terms dominate (the
    spectra, the indicator and the brick pool, about 37 bytes per voxel), it
    grows with points and mesh size, and bad arguments give -1."""
    from paper_1712_03084_gb300 import ftr
    e0 = ftr.ftr_estimate_bytes((256, 256, 256), 0, 0, 0, 0)
    assert 30 * 256 ** 3 < e0 < 45 * 256 ** 3
    e1 = ftr.ftr_estimate_bytes((256, 256, 256), 200000, 0, 100000, 200000)
    e2 = ftr.ftr_estimate_bytes((256, 256, 256), 400000, 0, 100000, 200000)
    assert e0 < e1 < e2
    assert ftr.ftr_estimate_bytes((256, 256, 256), 0, 0, 0, 0, ftr.FTR_PREC_BF16X3) > e0
    assert ftr.ftr_estimate_bytes((384, 384, 384), 0, 0, 0, 0) > 3 * e0
    with pytest.raises(ftr.FtrError):
        ftr.ftr_estimate_bytes((100, 256, 256), 0, 0, 0, 0)
    with pytest.raises(ftr.FtrError):
        ftr.ftr_estimate_bytes((256, 256, 256), -1, 0, 0, 0)


def test_estimate_per_point_terms_scale_with_the_frame(lib):
    """The point-dependent buffers (point store, (point, brick) pairs, work
    units, heavy-brick accumulators) follow the frame's point count: a
    10,000-point frame adds a few MB to a 96^3 context, not the tens of MB
    that accumulators sized for the minimum pair capacity would take, and a
    frame 16x larger adds about 16x as much."""
    from paper_1712_03084_gb300 import ftr
    g = (96, 96, 96)
    base = ftr.ftr_estimate_bytes(g, 0, 0, 0, 0)
    small = ftr.ftr_estimate_bytes(g, 10000, 0, 0, 0) - base
    big = ftr.ftr_estimate_bytes(g, 160000, 0, 0, 0) - base
    assert 0 < small < 8 << 20
    assert 8 * small < big < 32 * small


def test_marching_cubes_plan_arguments_are_checked_without_gpu(lib):
    """ftr_set_mc_plan takes two ints; the binding refuses other shapes before
    the library is called (the library's own range check needs a context)."""
    from paper_1712_03084_gb300 import ftr
    with pytest.raises(ValueError):
        ftr.ftr_set_mc_plan(None, (256,))
    with pytest.raises(ValueError):
        ftr.ftr_set_mc_plan(None, (256, 4, 1))
    assert lib.ftr_get_mc_plan(None, None) == -1      # FTR_EINVAL
    assert lib.ftr_set_mc_plan(None, None) == -1
