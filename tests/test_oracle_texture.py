"""Pins for the oracle per-vertex texture (Sec. III-C), no GPU.

The procedural texture is a smooth function of 3D position, so at a point on
the true surface that some camera sees, the blended colour must equal that
function up to bilinear and quantisation error; the UV must be the pixel
whose back-projected ray passes through the point (an independent form of
the projection); a point on the far side of the body is invisible.
"""

import numpy as np
import pytest

from datagen import human_frame
from datagen import scenes
from oracle import texture


@pytest.fixture(scope="module")
def small_frame():
    return human_frame(seed=3, depth_wh=(256, 212), fxy=182.5, rgb_wh=(480, 270), rgb_f=265.0)


def _surface_points(fr, cam_idx, n=400, seed=0):
    """True surface points seen by one depth camera (noise-free ray cast)."""
    cam = fr["cams"][cam_idx]
    rng = np.random.default_rng(seed)
    dw, _ = scenes.pixel_rays(cam)
    d = dw.reshape(-1, 3)
    t = scenes.raycast(fr["prims"], cam.pos, d)
    hit = np.nonzero(np.isfinite(t))[0]
    pick = rng.choice(hit, size=min(n, len(hit)), replace=False)
    return cam.pos + t[pick, None] * d[pick]


def test_uv_is_the_pixel_whose_ray_hits_the_point(small_frame):
    fr = small_frame
    X = _surface_points(fr, 0, 100)
    out = texture.texture(X, fr["views"], depth_tol=0.03)
    vw = fr["views"][0]
    Kr = vw["K_rgb"].astype(np.float64)
    RT = vw["world_to_rgb"].astype(np.float64)
    cpos = -RT[:, :3].T @ RT[:, 3]
    for i in np.nonzero(out["weights"][:, 0] > 0)[0]:
        u, v = out["uv"][i, 0]
        ray_c = np.array([(u - Kr[0, 2]) / Kr[0, 0], (v - Kr[1, 2]) / Kr[1, 1], 1.0])
        ray_w = RT[:, :3].T @ ray_c
        to_x = X[i] - cpos
        cosang = ray_w @ to_x / (np.linalg.norm(ray_w) * np.linalg.norm(to_x))
        assert cosang > 1 - 1e-6


def test_blended_colour_equals_the_surface_texture(small_frame):
    fr = small_frame
    X = np.concatenate([_surface_points(fr, k, 300, seed=k) for k in range(4)])
    out = texture.texture(X, fr["views"], depth_tol=0.03)
    ok = out["textured"] == 1
    assert ok.mean() > 0.5
    truth = scenes.procedural_colour(X, fr["texture_params"])
    err = np.abs(out["rgb"][ok].astype(float) - truth[ok])
    # bilinear sampling of a texture with >= 0.12 m wavelength at ~1 cm pixels
    assert np.median(err) < 6.0
    assert np.percentile(err, 90) < 25.0


def test_far_side_is_invisible(small_frame):
    fr = small_frame
    X = _surface_points(fr, 0, 200)
    out = texture.texture(X, fr["views"], depth_tol=0.03)
    # camera 2 sits opposite camera 0 on the ring: it must not see camera 0's
    # surface points that lie behind the body centre as seen from camera 2
    cam0, cam2 = fr["cams"][0], fr["cams"][2]
    c = np.array([0.0, 0.95, 0.0])
    behind = ((X - c) @ (cam0.pos - c)) > 0.12
    assert np.all(out["weights"][behind, 2] == 0)
    assert np.all(out["uv"][behind, 2] == -1)
    assert cam2 is not None


def test_weights_equal_confidence_at_nearest_pixel(small_frame):
    fr = small_frame
    X = _surface_points(fr, 1, 200)
    out = texture.texture(X, fr["views"], depth_tol=0.03)
    vw = fr["views"][1]
    u, v, z = texture.project(vw["K"], vw["world_to_cam"], X)
    px = np.floor(u + 0.5).astype(int)
    py = np.floor(v + 0.5).astype(int)
    vis = out["weights"][:, 1] > 0
    assert vis.mean() > 0.5
    assert np.allclose(out["weights"][vis, 1], vw["conf"][py[vis], px[vis]])
