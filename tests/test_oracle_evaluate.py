"""Pins of the oracle's evaluation metrics (Sec. III-E, eq. (3)-(7)):
closed forms on simple silhouettes and images, the missing-limb and hole
cases the paper describes for eq. (4), independent library routines (an exact
Euclidean distance transform, a k-d tree, a library correlation) on random
inputs, and the paper's WMS3IM constants."""

import json
import os

import numpy as np
import pytest

from oracle import evaluate as ev

K = np.array([[100.0, 0.0, 32.0], [0.0, 100.0, 24.0], [0.0, 0.0, 1.0]], np.float32)


def _mask_depth(mask, z=2.0):
    return np.where(mask, np.float32(z), np.float32(0.0))


def test_vre_closed_forms():
    a = np.zeros((40, 60), bool)
    b = np.zeros((40, 60), bool)
    a[5:25, 10:30] = True        # 400 px
    b[15:35, 20:40] = True       # 400 px, overlap 10 x 10
    v, x, o, nr, ng = ev.vre(_mask_depth(a), _mask_depth(b))
    assert (x, o, nr, ng) == (600, 700, 400, 400) and v == pytest.approx(600 / 700)
    assert ev.vre(_mask_depth(a), _mask_depth(a))[0] == 0.0
    c = np.zeros_like(a)
    c[30:38, 45:55] = True
    assert ev.vre(_mask_depth(a), _mask_depth(c))[0] == 1.0
    assert ev.vre(_mask_depth(c & False), _mask_depth(c & False))[0] == 0.0


def test_hausdorff_closed_forms_and_the_papers_cases():
    a = np.zeros((30, 30), bool)
    b = np.zeros((30, 30), bool)
    a[2, 3] = True
    b[6, 6] = True
    assert ev.hausdorff(_mask_depth(a), _mask_depth(b)) == 5.0
    # missing limb: a 25-pixel arm left out of the reconstruction
    body = np.zeros((80, 80), bool)
    body[20:60, 20:40] = True
    gt = body.copy()
    gt[30:33, 40:65] = True
    assert ev.hausdorff(_mask_depth(body), _mask_depth(gt)) == 25.0
    # hole: the distance is the radius of the inscribed circle; for the pixels
    # within 6 of the centre the nearest pixel outside lies at offset (6, 1)
    jj, ii = np.mgrid[0:80, 0:80]
    hole = (jj - 40) ** 2 + (ii - 40) ** 2 <= 36
    full = np.zeros((80, 80), bool)
    full[10:70, 10:70] = True
    assert ev.hausdorff(_mask_depth(full & ~hole), _mask_depth(full)) == np.sqrt(37.0)
    assert ev.hausdorff(_mask_depth(a & False), _mask_depth(b)) == float("inf")
    assert ev.hausdorff(_mask_depth(a & False), _mask_depth(a & False)) == 0.0


def test_hausdorff_equals_the_exact_distance_transform():
    from scipy import ndimage
    rng = np.random.default_rng(4)
    for _ in range(3):
        r = ndimage.binary_dilation(rng.random((50, 70)) > 0.985, iterations=3)
        g = ndimage.binary_dilation(rng.random((50, 70)) > 0.985, iterations=2)
        d_to_g = ndimage.distance_transform_edt(~g)
        d_to_r = ndimage.distance_transform_edt(~r)
        want = max(d_to_g[r].max(), d_to_r[g].max())
        assert ev.hausdorff(_mask_depth(r), _mask_depth(g)) == pytest.approx(want, abs=1e-12)


def test_cp_rmse_closed_form_and_kdtree():
    from scipy.spatial import cKDTree
    gt = np.zeros((48, 64), np.float32)
    rec = np.zeros((48, 64), np.float32)
    gt[10, 20] = 2.0
    rec[10, 20] = 2.5
    rmse, I, J = ev.cp_rmse(K, rec, gt)
    dx, dy = (20 - 32.0) / 100.0, (10 - 24.0) / 100.0
    assert (I, J) == (1, 1) and rmse == pytest.approx(0.5 * np.sqrt(dx * dx + dy * dy + 1), rel=1e-12)
    assert ev.cp_rmse(K, gt, gt)[0] == 0.0
    rng = np.random.default_rng(7)
    g = np.where(rng.random((48, 64)) > 0.6, rng.uniform(1.5, 3, (48, 64)), 0).astype(np.float32)
    r = np.where(rng.random((48, 64)) > 0.5, rng.uniform(1.5, 3, (48, 64)), 0).astype(np.float32)
    rmse, I, J = ev.cp_rmse(K, r, g)
    Xg, Xr = ev.backproject(K, g), ev.backproject(K, r)
    d, _ = cKDTree(Xr).query(Xg)
    assert rmse == pytest.approx(np.sqrt(np.mean(d * d)), rel=1e-12)
    assert np.isnan(ev.cp_rmse(K, r, g * 0)[0]) and ev.cp_rmse(K, r * 0, g)[0] == float("inf")


def test_window_mean_is_the_normalised_library_correlation():
    from scipy import ndimage
    rng = np.random.default_rng(2)
    img = rng.uniform(0, 255, (37, 53))
    g = ev.gaussian_taps()
    k2 = np.outer(g, g)
    want = ndimage.correlate(img, k2, mode="constant") / ndimage.correlate(np.ones_like(img), k2, mode="constant")
    assert np.max(np.abs(ev.window_mean(img, g) - want)) < 1e-10
    m = rng.random((37, 53)) > 0.5
    cnt = ndimage.correlate(m.astype(np.int64), np.ones((11, 11), np.int64), mode="constant")
    assert np.array_equal(ev.window_count(m), cnt)
    # images smaller than the window
    for shape in ((3, 3), (1, 7), (6, 2)):
        img = rng.uniform(0, 255, shape)
        want = ndimage.correlate(img, k2, mode="constant") / ndimage.correlate(np.ones_like(img), k2, mode="constant")
        assert np.max(np.abs(ev.window_mean(img, g) - want)) < 1e-10
        m = rng.random(shape) > 0.3
        cnt = ndimage.correlate(m.astype(np.int64), np.ones((11, 11), np.int64), mode="constant")
        assert np.array_equal(ev.window_count(m), cnt)


def _grey(v):
    v = np.asarray(v, np.uint8)
    return np.stack([v, v, v], -1)


def test_wms3im_closed_forms():
    rng = np.random.default_rng(3)
    img = rng.integers(0, 256, (64, 96, 3)).astype(np.uint8)
    mask = np.zeros((64, 96), bool)
    mask[8:56, 10:80] = True
    d = _mask_depth(mask)
    out, L, C, S = ev.wms3im(d, img, img)
    assert out == pytest.approx(1.0, abs=1e-12)
    assert np.allclose(L + C + S, 1.0, atol=1e-12)
    # constant images: only the luminance term of scale 3 is below 1
    a, b = 90.0, 150.0
    out, L, C, S = ev.wms3im(d, _grey(np.full((64, 96), a)), _grey(np.full((64, 96), b)))
    lum = (2 * a * b + ev.SSIM_C1) / (a * a + b * b + ev.SSIM_C1)
    assert np.allclose(C + S, 1.0, atol=1e-9) and np.allclose(L, lum, rtol=1e-9)
    assert out == pytest.approx(lum ** 0.1333, rel=1e-9)
    # a positive linear map keeps the structure term at 1 on every scale
    x = rng.integers(0, 120, (64, 96))
    out, L, C, S = ev.wms3im(d, _grey(x), _grey(2 * x + 3))
    assert np.allclose(S, 1.0, atol=1e-6) and all(c < 1 for c in C)
    # inverted contrast: negative structure, no real power, WMS3IM = 0
    out, L, C, S = ev.wms3im(d, _grey(x + 60), _grey(195 - x))
    assert min(S) < 0 and out == 0.0
    # symmetric in the two images
    y = rng.integers(0, 256, (64, 96, 3)).astype(np.uint8)
    assert ev.wms3im(d, img, y)[0] == pytest.approx(ev.wms3im(d, y, img)[0], rel=1e-12)
    assert np.isnan(ev.wms3im(d * 0, img, y)[0])


def test_scales_and_the_papers_constants():
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")) as f:
        pc = json.load(f)
    assert list(ev.WMS3IM_ALPHA) == pc["wms3im_alpha"]["value"]
    assert list(ev.WMS3IM_BETA) == pc["wms3im_beta_gamma"]["value"]
    assert list(ev.WMS3IM_GAMMA) == pc["wms3im_beta_gamma"]["value"]
    X = np.arange(7 * 9, dtype=float).reshape(7, 9)
    S = np.ones((7, 9), bool)
    S[0, 0] = False
    Xn, Sn = ev.downsample(X, S)
    assert Xn.shape == (3, 4) and Xn[1, 2] == np.mean(X[2:4, 4:6]) and not Sn[0, 0] and Sn[1:, :].all()
