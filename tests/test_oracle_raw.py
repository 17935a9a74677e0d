"""Pins of the raw-reconstruction oracle (Sec. III-A): back-projection,
organised-triangulation normals, confidence weights."""

import numpy as np

from oracle import conventions as cv
from oracle import raw

K = np.array([[180.0, 0.0, 63.5], [0.0, 170.0, 47.5], [0.0, 0.0, 1.0]])


def plane_depth(n, d, h=96, w=128, Kc=K):
    """Depth map of the plane n . x = d seen by a camera at the origin."""
    v, u = np.meshgrid(np.arange(h, dtype=np.float64), np.arange(w, dtype=np.float64), indexing="ij")
    ray = np.stack([(u - Kc[0, 2]) / Kc[0, 0], (v - Kc[1, 2]) / Kc[1, 1], np.ones_like(u)], axis=-1)
    return d / (ray @ np.asarray(n, dtype=np.float64))


def test_back_projection_reprojects_to_the_pixel():
    rng = np.random.default_rng(0)
    D = rng.uniform(0.5, 3.0, (40, 50))
    xc = raw.camera_points(D, K)
    u = K[0, 0] * xc[..., 0] / xc[..., 2] + K[0, 2]
    v = K[1, 1] * xc[..., 1] / xc[..., 2] + K[1, 2]
    jj, ii = np.meshgrid(np.arange(40), np.arange(50), indexing="ij")
    assert np.allclose(u, ii, atol=1e-10) and np.allclose(v, jj, atol=1e-10)
    assert np.array_equal(xc[..., 2], D)


def test_world_transform_inverts_the_extrinsics():
    rng = np.random.default_rng(1)
    q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    R = q * np.sign(np.linalg.det(q))
    t = rng.standard_normal(3)
    RT = np.concatenate([R, t[:, None]], axis=1)
    D = plane_depth([0.1, -0.2, 1.0], 2.0)
    P, N, W, _ = raw.raw_points(D, K, RT)
    xc = raw.camera_points(D, K)
    mask = np.ones(D.shape, bool)
    assert np.allclose(P @ R.T + t, xc[mask], atol=1e-12)


def test_plane_normals_and_w1_closed_form():
    n = np.array([0.2, -0.3, 1.0])
    n /= np.linalg.norm(n)
    D = plane_depth(n, 2.0)
    xc = raw.camera_points(D, K)
    nc, mask = raw.vertex_normals(xc, D)
    assert mask.all()
    facing = -n if n[2] > 0 else n          # toward the camera at the origin
    assert np.abs(nc - facing).max() < 1e-9
    P, N, W, Wmap = raw.raw_points(D, K, np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1))
    xhat = -xc / np.linalg.norm(xc, axis=-1, keepdims=True)
    w1 = np.maximum(xhat @ facing, 0.0)
    w2 = raw.silhouette_mean(D)
    assert np.abs(Wmap - w1 * w2).max() < 1e-9


def test_depth_step_splits_the_triangulation():
    D = np.full((30, 40), 1.0)
    D[:, 20:] = 2.0                            # 1 m step: far above 0.03 + 3 * 0.0012 * 4
    xc = raw.camera_points(D, K)
    tri = raw.triangle_normals(xc, D)
    for corners, keep, n in tri:
        cols = [b for (_, b) in corners]
        # quads whose corners reach both sides (top-left column 19) keep nothing
        assert not keep[:, 19].any()
        assert keep[:, :19].all() and keep[:, 20:].all()
    nc, mask = raw.vertex_normals(xc, D)
    assert mask.all()
    assert np.abs(nc - np.array([0.0, 0.0, -1.0])).max() < 1e-12    # fronto-parallel on both sides
    # a step within the threshold is kept
    D2 = D.copy()
    D2[:, 20:] = 1.0 + 0.5 * (cv.TSDC_STEP + 3.0 * cv.TSDC_NOISE)
    keep2 = raw.triangle_normals(raw.camera_points(D2, K), D2)[0][1]
    assert keep2[:, 19].all()


def test_isolated_and_background_pixels_give_no_point():
    D = np.zeros((20, 20))
    D[5, 5] = 1.0                              # a lone foreground pixel: no triangle
    D[10:12, 10:12] = 1.5                      # one quad: two triangles
    P, N, W, Wmap = raw.raw_points(D, K, np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1))
    assert len(P) == 4
    assert Wmap[5, 5] == 0.0 and (Wmap[D == 0] == 0).all()


def test_silhouette_mean_border_values_and_summed_area_table():
    r = cv.W2_RADIUS
    m = np.ones((50, 60))
    w2 = raw.silhouette_mean(m)
    k = 2 * r + 1
    assert w2[25, 30] == 1.0
    assert abs(w2[0, 0] - (r + 1) ** 2 / k ** 2) < 1e-15
    assert abs(w2[0, 30] - (r + 1) / k) < 1e-15
    rng = np.random.default_rng(2)
    mask = rng.random((37, 41)) < 0.4
    sat = np.zeros((37 + 1, 41 + 1))
    sat[1:, 1:] = mask.cumsum(0).cumsum(1)
    y0 = np.clip(np.arange(37) - r, 0, 37)
    y1 = np.clip(np.arange(37) + r + 1, 0, 37)
    x0 = np.clip(np.arange(41) - r, 0, 41)
    x1 = np.clip(np.arange(41) + r + 1, 0, 41)
    ref = (sat[y1][:, x1] - sat[y0][:, x1] - sat[y1][:, x0] + sat[y0][:, x0]) / k ** 2
    assert np.abs(raw.silhouette_mean(mask) - ref).max() < 1e-15


def test_matches_the_input_generator_on_a_human_view():
    """An independent implementation (the synthetic-input generator's) on the
    same float32 depth map gives the same points, normals and weights."""
    from datagen import human_frame
    from datagen import scenes
    fr = human_frame(seed=3, depth_wh=(256, 212), fxy=182.5, with_rgb=False)
    cam = fr["cams"][0]
    D = fr["views"][0]["depth"].astype(np.float64)
    xc, xw = scenes.backproject(cam, D)
    nc, valid = scenes.organised_normals(xc, D)
    P, N, W, Wmap = raw.raw_points(fr["views"][0]["depth"], cam.K, cam.world_to_cam)
    assert len(P) == int(valid.sum())
    assert np.abs(P - xw[valid]).max() < 1e-9
    assert np.abs(N - (nc @ cam.R)[valid]).max() < 1e-9
    xhat = -xc / np.maximum(np.linalg.norm(xc, axis=-1, keepdims=True), 1e-12)
    w = np.maximum(np.sum(xhat * nc, axis=-1), 0.0) * scenes.box_mean(D > 0, cv.W2_RADIUS)
    assert np.abs(W - w[valid]).max() < 1e-12
