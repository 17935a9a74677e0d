"""The texture stage takes its decisions (nearest depth pixel, depth test,
RGB bounds) in float32 and re-decides in float64 only inside guard bands of
2e-3 px and 1e-4 m.  That is sound only if float32 evaluation errs by much
less than the bands: measured here on the CPU, emulating the float32
projection operation by operation (each product and sum rounded to float32,
the order of the kernel's expression), over a million random vertices in the
human frame's box seen by every camera of the frame."""

import numpy as np

from datagen import frame_config, human_frame


def _project_f32(K, RT, X):
    f = np.float32
    K = K.astype(f).reshape(-1)
    RT = RT.astype(f).reshape(-1)
    X = X.astype(f)

    def dot3(r0, r1, r2, t):
        # ((r0 x + r1 y) + r2 z) + t, every step rounded to float32
        return (((r0 * X[:, 0]).astype(f) + (r1 * X[:, 1]).astype(f)).astype(f)
                + (r2 * X[:, 2]).astype(f)).astype(f) + f(t)
    xc = dot3(RT[0], RT[1], RT[2], RT[3]).astype(f)
    yc = dot3(RT[4], RT[5], RT[6], RT[7]).astype(f)
    zc = dot3(RT[8], RT[9], RT[10], RT[11]).astype(f)
    uu = ((K[0] * xc + K[1] * yc).astype(f) + (K[2] * zc).astype(f)).astype(f)
    vv = ((K[3] * xc + K[4] * yc).astype(f) + (K[5] * zc).astype(f)).astype(f)
    ww = ((K[6] * xc + K[7] * yc).astype(f) + (K[8] * zc).astype(f)).astype(f)
    return (uu / ww).astype(f), (vv / ww).astype(f), zc


def _project_f64(K, RT, X):
    K = K.astype(np.float32).astype(np.float64).reshape(3, 3)
    RT = RT.astype(np.float32).astype(np.float64).reshape(3, 4)
    X = X.astype(np.float32).astype(np.float64)
    xc = X @ RT[:, :3].T + RT[:, 3]
    uvw = xc @ K.T
    return uvw[:, 0] / uvw[:, 2], uvw[:, 1] / uvw[:, 2], xc[:, 2]


def test_float32_errors_are_far_inside_the_texture_guard_bands():
    cfg = frame_config("human256")
    # the rig (camera poses) of the human256 frame; small images suffice for the poses
    fr = human_frame(seed=1, K=cfg["K"], ring=cfg["ring"], height=cfg["height"],
                     depth_wh=(64, 53), fxy=45.6, rgb_wh=(32, 18), rgb_f=35.0)
    rng = np.random.default_rng(0)
    lo, hi = np.array(cfg["bbox"][:3]), np.array(cfg["bbox"][3:])
    X = (lo + (hi - lo) * rng.random((1_000_000, 3))).astype(np.float32)
    # the full-size intrinsics of the frame's cameras (512 x 424, f = 365; 1920 x 1080, f = 1060)
    Kd = np.array([[365.0, 0, 256.0], [0, 365.0, 212.0], [0, 0, 1.0]])
    Kc = np.array([[1060.0, 0, 960.0], [0, 1060.0, 540.0], [0, 0, 1.0]])
    worst_px, worst_m = 0.0, 0.0
    for v in fr["views"]:
        for K, RT in ((Kd, v["world_to_cam"]), (Kc, v["world_to_rgb"])):
            u32, v32, z32 = _project_f32(K, RT, X)
            u64, v64, z64 = _project_f64(K, RT, X)
            front = z64 > 0.5
            worst_px = max(worst_px, float(np.max(np.abs(u32[front] - u64[front]))),
                           float(np.max(np.abs(v32[front] - v64[front]))))
            worst_m = max(worst_m, float(np.max(np.abs(z32 - z64))))
    assert worst_px < 2e-3 / 4, worst_px          # pixel band 2e-3 px
    assert worst_m < 1e-4 / 4, worst_m            # depth band 1e-4 m
