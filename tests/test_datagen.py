"""The seeded input generator is deterministic and produces sane inputs (no GPU)."""

import numpy as np

from datagen import human_frame, sphere_points


def test_sphere_is_seeded():
    a = sphere_points(1000, 0.005, seed=0)
    b = sphere_points(1000, 0.005, seed=0)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert a[0].dtype == np.float32
    assert np.allclose(np.linalg.norm(a[1], axis=1), 1.0, atol=1e-6)


def test_human_frame_is_seeded_and_sane():
    kw = dict(depth_wh=(128, 106), fxy=91.25, with_rgb=False)
    a = human_frame(seed=5, **kw)
    b = human_frame(seed=5, **kw)
    assert np.array_equal(a["points"], b["points"])
    assert np.array_equal(a["weights"], b["weights"])
    P = a["points"]
    assert len(P) > 1000
    assert np.all(P[:, 1] > -0.05) and np.all(P[:, 1] < 1.95)
    assert np.allclose(np.linalg.norm(a["normals"], axis=1), 1.0, atol=1e-5)
    assert np.all((a["weights"] >= 0) & (a["weights"] <= 1))
    # normals face their camera (W1 > 0 wherever W > 0)
    for (s, n), cam in zip(a["per_camera"], a["cams"]):
        d = cam.pos - P[s:s + n]
        assert np.mean(np.einsum("ij,ij->i", d, a["normals"][s:s + n]) > 0) > 0.99


def test_pose_seed_moves_the_body_not_the_rig():
    from datagen import human_frame
    kw = dict(K=2, depth_wh=(64, 53), fxy=45.6, rgb_wh=(32, 18), rgb_f=35.0)
    a = human_frame(seed=5, **kw)
    b = human_frame(seed=5, pose_seed=99, **kw)
    for va, vb in zip(a["views"], b["views"]):
        assert np.array_equal(va["K"], vb["K"]) and np.array_equal(va["world_to_cam"], vb["world_to_cam"])
        assert np.array_equal(va["world_to_rgb"], vb["world_to_rgb"])
    assert not np.array_equal(a["views"][0]["depth"], b["views"][0]["depth"])
