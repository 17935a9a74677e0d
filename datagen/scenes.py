"""Synthetic scenes: a noisy sphere and a multi-camera capsule human.

Inputs only (see ``datagen/__init__``).  All randomness comes from
``numpy.random.default_rng(seed)``.

Sphere: n points uniform on the unit sphere (normalised Gaussian triples),
exact outward normals, positions perturbed by isotropic Gaussian noise,
unit weights.

Human frame: an articulated body of 15 capsules/ellipsoids (~1.8 m tall)
with seeded joint angles, seen by K depth cameras on a ring looking at the
body.  Per camera: analytic ray cast of every depth pixel, depth noise
sigma = 0.0012 z^2, back-projection of foreground pixels, normals from an
organised triangulation (two triangles per 2x2 pixel quad, skipped across a
depth step), W1 = max(<-X^, N>, 0), W2 = 21x21 box mean of the silhouette,
W = W1 W2 (Sec. III-A).  RGB views come from a second ray cast through an
RGB camera offset 5 cm sideways, coloured by a seeded smooth procedural
texture of the 3D hit position.
"""

from dataclasses import dataclass, field

import numpy as np


# --------------------------------------------------------------------------- sphere

def sphere_points(n=20000, noise=0.005, seed=0, radius=1.0):
    """Points on a sphere of ``radius`` with outward normals; returns float32 arrays."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((n, 3))
    nrm = g / np.linalg.norm(g, axis=1, keepdims=True)
    pts = radius * nrm + noise * rng.standard_normal((n, 3))
    w = np.ones(n)
    return pts.astype(np.float32), nrm.astype(np.float32), w.astype(np.float32)


# --------------------------------------------------------------------------- cameras

@dataclass
class Camera:
    w: int
    h: int
    K: np.ndarray            # 3x3
    world_to_cam: np.ndarray  # 3x4 [R | t]
    pos: np.ndarray          # camera centre (world)

    @property
    def R(self):
        return self.world_to_cam[:, :3]


def look_at(pos, target, up=(0.0, 1.0, 0.0)):
    """Rows (right, down, forward) of a camera at pos looking at target."""
    pos = np.asarray(pos, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - pos
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, dtype=np.float64))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    return np.stack([r, d, f])


def make_camera(pos, target, w, h, fx, fy, cx=None, cy=None):
    R = look_at(pos, target)
    t = -R @ np.asarray(pos, dtype=np.float64)
    K = np.array([[fx, 0.0, (w / 2.0) if cx is None else cx],
                  [0.0, fy, (h / 2.0) if cy is None else cy],
                  [0.0, 0.0, 1.0]])
    return Camera(w, h, K, np.concatenate([R, t[:, None]], axis=1), np.asarray(pos, float))


def ring_cameras(K=4, radius=2.5, height=1.2, target=(0.0, 0.95, 0.0), w=512, h=424,
                 fx=365.0, fy=365.0, phase_deg=0.0):
    """K cameras evenly spaced on a ring, all looking at ``target``."""
    cams = []
    for k in range(K):
        th = np.deg2rad(phase_deg + 360.0 * k / K)
        pos = (target[0] + radius * np.sin(th), height, target[2] + radius * np.cos(th))
        cams.append(make_camera(pos, target, w, h, fx, fy))
    return cams


def rgb_companion(cam, w=1920, h=1080, fx=1060.0, fy=1060.0, offset=0.05):
    """RGB camera parallel to the depth camera, shifted ``offset`` m along its x axis."""
    R = cam.R
    pos = cam.pos + offset * R[0]
    t = -R @ pos
    K = np.array([[fx, 0.0, w / 2.0], [0.0, fy, h / 2.0], [0.0, 0.0, 1.0]])
    return Camera(w, h, K, np.concatenate([R, t[:, None]], axis=1), pos)


def pixel_rays(cam):
    """World-space unit ray directions [h, w, 3] and the cosine to the optical axis."""
    jj, ii = np.meshgrid(np.arange(cam.h, dtype=np.float64),
                         np.arange(cam.w, dtype=np.float64), indexing="ij")
    dc = np.stack([(ii - cam.K[0, 2]) / cam.K[0, 0],
                   (jj - cam.K[1, 2]) / cam.K[1, 1],
                   np.ones_like(ii)], axis=-1)
    nrm = np.linalg.norm(dc, axis=-1, keepdims=True)
    dc = dc / nrm
    dw = dc @ cam.R          # R^T d for row vectors
    return dw, dc[..., 2]


# --------------------------------------------------------------------------- body

@dataclass
class Capsule:
    a: np.ndarray
    b: np.ndarray
    r: float


@dataclass
class Ellipsoid:
    c: np.ndarray
    radii: np.ndarray
    R: np.ndarray = field(default_factory=lambda: np.eye(3))   # rows: local axes


def _rot(axis, deg):
    th = np.deg2rad(deg)
    c, s = np.cos(th), np.sin(th)
    if axis == "x":
        return np.array([[1, 0, 0], [0, c, -s], [0, s, c]])
    if axis == "y":
        return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]])
    return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]])


def human_primitives(seed=0, angle_range=40.0, yaw_deg=None):
    """15 primitives of a ~1.8 m human; joint angles drawn uniformly in +-angle_range."""
    rng = np.random.default_rng(seed)

    def ang(lo, hi):
        return float(rng.uniform(lo, hi))

    prims = []
    prims.append(Ellipsoid(np.array([0.0, 1.665, 0.0]), np.array([0.085, 0.115, 0.100])))  # head
    prims.append(Ellipsoid(np.array([0.0, 1.23, 0.0]), np.array([0.175, 0.27, 0.115])))    # torso
    prims.append(Ellipsoid(np.array([0.0, 0.95, 0.0]), np.array([0.160, 0.115, 0.105])))   # pelvis
    ar = angle_range
    for side in (-1.0, 1.0):
        # arm: hangs down at rest; abduction about z, flexion about x, elbow about x
        sh = np.array([side * 0.205, 1.44, 0.0])
        abd = 20.0 + ang(-0.5 * ar, ar)
        flex = ang(-ar, ar)
        elb = ang(0.0, 2.0 * ar)
        Ru = _rot("x", -flex) @ _rot("z", side * abd)
        du = Ru @ np.array([0.0, -1.0, 0.0])
        el = sh + 0.29 * du
        df = _rot("x", -elb) @ du
        df /= np.linalg.norm(df)
        wr = el + 0.26 * df
        prims.append(Capsule(sh, el, 0.047))
        prims.append(Capsule(el, wr, 0.038))
        hc = wr + 0.085 * df
        prims.append(Ellipsoid(hc, np.array([0.045, 0.085, 0.022]), _frame_from_dir(df)))
        # leg: hip flexion about x, abduction about z, knee bends backwards
        hp = np.array([side * 0.09, 0.90, 0.0])
        hflex = ang(-0.6 * ar, 0.6 * ar)
        habd = ang(0.0, 0.3 * ar)
        knee = ang(0.0, 1.2 * ar)
        Rl = _rot("x", -hflex) @ _rot("z", side * habd)
        dt = Rl @ np.array([0.0, -1.0, 0.0])
        kn = hp + 0.42 * dt
        ds = _rot("x", knee) @ dt
        ds /= np.linalg.norm(ds)
        an = kn + 0.41 * ds
        prims.append(Capsule(hp, kn, 0.072))
        prims.append(Capsule(kn, an, 0.053))
        fwd = np.array([0.0, 0.0, 1.0])
        prims.append(Ellipsoid(an + np.array([0.0, -0.035, 0.055]),
                               np.array([0.045, 0.035, 0.120]), _frame_from_dir(fwd)))
    yaw = ang(-180.0, 180.0) if yaw_deg is None else yaw_deg
    Ry = _rot("y", yaw)
    pivot = np.array([0.0, 0.95, 0.0])
    out = []
    for p in prims:
        if isinstance(p, Capsule):
            out.append(Capsule(Ry @ (p.a - pivot) + pivot, Ry @ (p.b - pivot) + pivot, p.r))
        else:
            out.append(Ellipsoid(Ry @ (p.c - pivot) + pivot, p.radii, p.R @ Ry.T))
    assert len(out) == 15
    return out


def _frame_from_dir(d):
    """Rows of an orthonormal frame whose second row is the unit direction d."""
    d = d / np.linalg.norm(d)
    ref = np.array([1.0, 0.0, 0.0]) if abs(d[0]) < 0.9 else np.array([0.0, 0.0, 1.0])
    a = np.cross(ref, d)
    a /= np.linalg.norm(a)
    c = np.cross(a, d)
    return np.stack([a, d, c])


def _ray_sphere(o, d, c, r):
    oc = o - c
    b = oc @ d if oc.ndim == 1 else np.einsum("ij,ij->i", oc, d)
    cc = np.sum(oc * oc, axis=-1) - r * r
    disc = b * b - cc
    with np.errstate(invalid="ignore"):
        t = -b - np.sqrt(disc)
    return np.where(disc >= 0, t, np.inf)


def _ray_capsule(o, d, cap):
    """First hit distance of rays o + t d (d unit) with a capsule (inf on a miss)."""
    ba = cap.b - cap.a
    L2 = ba @ ba
    u = ba / np.sqrt(L2)
    oa = o - cap.a
    du = d @ u
    ou = oa @ u if oa.ndim == 1 else oa @ u
    dp = d - du[:, None] * u
    op = oa - (ou[:, None] * u if np.ndim(ou) else ou * u)
    A = np.sum(dp * dp, axis=-1)
    B = np.sum(dp * op, axis=-1)
    C = np.sum(op * op, axis=-1) - cap.r ** 2
    disc = B * B - A * C
    with np.errstate(invalid="ignore", divide="ignore"):
        t = (-B - np.sqrt(disc)) / A
    y = ou + t * du
    L = np.sqrt(L2)
    tc = np.where((disc >= 0) & (A > 1e-12) & (y >= 0) & (y <= L), t, np.inf)
    t1 = _ray_sphere(o, d, cap.a, cap.r)
    t2 = _ray_sphere(o, d, cap.b, cap.r)
    t = np.minimum(tc, np.minimum(t1, t2))
    return np.where(t > 1e-6, t, np.inf)


def _ray_ellipsoid(o, d, el):
    M = el.R / el.radii[:, None]           # maps world offset to unit-sphere coords
    op = (o - el.c) @ M.T
    dp = d @ M.T
    a = np.sum(dp * dp, axis=-1)
    b = np.sum(op * dp, axis=-1)
    c = np.sum(op * op, axis=-1) - 1.0
    disc = b * b - a * c
    with np.errstate(invalid="ignore"):
        t = (-b - np.sqrt(disc)) / a
    return np.where((disc >= 0) & (t > 1e-6), t, np.inf)


def raycast(prims, origin, dirs, device=None):
    """Nearest hit distance along unit rays from one origin (inf on a miss).

    ``device`` (e.g. "cuda") evaluates the same intersections with torch."""
    if device is not None:
        from .torch_raycast import raycast_torch
        return raycast_torch(prims, origin, dirs, device)
    o = np.asarray(origin, dtype=np.float64)
    best = np.full(len(dirs), np.inf)
    for p in prims:
        if isinstance(p, Capsule):
            t = _ray_capsule(np.broadcast_to(o, dirs.shape), dirs, p)
        else:
            t = _ray_ellipsoid(o, dirs, p)
        best = np.minimum(best, t)
    return best


# --------------------------------------------------------------------------- depth views

def depth_view(cam, prims, rng, noise_coef=0.0012, device=None):
    """Noisy depth map (0 = background) of the body seen by ``cam``."""
    dw, cosax = pixel_rays(cam)
    t = raycast(prims, cam.pos, dw.reshape(-1, 3), device).reshape(cam.h, cam.w)
    fg = np.isfinite(t)
    z = np.where(fg, t * cosax, 0.0)
    sig = noise_coef * z * z
    z = np.where(fg, z + sig * rng.standard_normal(z.shape), 0.0)
    return z


def backproject(cam, z):
    """Camera- and world-space points [h, w, 3] of a depth map."""
    jj, ii = np.meshgrid(np.arange(cam.h, dtype=np.float64),
                         np.arange(cam.w, dtype=np.float64), indexing="ij")
    xc = np.stack([(ii - cam.K[0, 2]) / cam.K[0, 0] * z,
                   (jj - cam.K[1, 2]) / cam.K[1, 1] * z, z], axis=-1)
    xw = (xc - cam.world_to_cam[:, 3]) @ cam.R       # R^T (xc - t)
    return xc, xw


def organised_normals(xc, z, noise_coef=0.0012, step=0.03):
    """Camera-space vertex normals from two triangles per 2x2 quad (depth-step test)."""
    h, w = z.shape
    fg = z > 0
    acc = np.zeros((h, w, 3))
    cnt = np.zeros((h, w))
    p00, p10, p01, p11 = xc[:-1, :-1], xc[:-1, 1:], xc[1:, :-1], xc[1:, 1:]
    z00, z10, z01, z11 = z[:-1, :-1], z[:-1, 1:], z[1:, :-1], z[1:, 1:]
    f00, f10, f01, f11 = fg[:-1, :-1], fg[:-1, 1:], fg[1:, :-1], fg[1:, 1:]
    zmax = np.maximum(np.maximum(z00, z10), np.maximum(z01, z11))
    thr = step + 3.0 * noise_coef * zmax * zmax
    tris = (((p00, p10, p01), (z00, z10, z01), (f00, f10, f01),
             ((slice(0, -1), slice(0, -1)), (slice(0, -1), slice(1, None)), (slice(1, None), slice(0, -1)))),
            ((p10, p11, p01), (z10, z11, z01), (f10, f11, f01),
             ((slice(0, -1), slice(1, None)), (slice(1, None), slice(1, None)), (slice(1, None), slice(0, -1)))))
    for (a, b, c), (za, zb, zc), (fa, fb, fc), sl in tris:
        ok = fa & fb & fc
        dz = np.maximum(np.maximum(np.abs(za - zb), np.abs(zb - zc)), np.abs(za - zc))
        ok &= dz <= thr
        n = np.cross(b - a, c - a)
        ln = np.linalg.norm(n, axis=-1)
        ok &= ln > 0
        n = np.where(ok[..., None], n / np.where(ln > 0, ln, 1.0)[..., None], 0.0)
        cen = (a + b + c) / 3.0
        flip = np.sum(n * cen, axis=-1) > 0        # orient toward the camera at the origin
        n = np.where(flip[..., None], -n, n)
        for s in sl:
            acc[s] += n
            cnt[s] += ok
    ln = np.linalg.norm(acc, axis=-1)
    valid = fg & (cnt > 0) & (ln > 0)
    nrm = np.where(valid[..., None], acc / np.where(ln > 0, ln, 1.0)[..., None], 0.0)
    return nrm, valid


def box_mean(mask, radius=10):
    """Mean of a binary image over a (2r+1)^2 window, zero outside (Sec. III-A W2)."""
    m = mask.astype(np.float64)
    h, w = m.shape
    k = 2 * radius + 1
    pad = np.zeros((h + 2 * radius + 1, w + 2 * radius + 1))
    pad[radius + 1:radius + 1 + h, radius + 1:radius + 1 + w] = m
    s = pad.cumsum(0).cumsum(1)
    out = s[k:k + h, k:k + w] - s[0:h, k:k + w] - s[k:k + h, 0:w] + s[0:h, 0:w]
    return out / (k * k)


# --------------------------------------------------------------------------- RGB views

def texture_params(seed):
    rng = np.random.default_rng(seed + 7919)
    dirs = rng.standard_normal((3, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    lam = rng.uniform(0.12, 0.35, 3)
    phase = rng.uniform(0.0, 2.0 * np.pi, 3)
    return dirs, lam, phase


def procedural_colour(X, params):
    """Smooth RGB in [28, 228] as a function of the 3D position (float64)."""
    dirs, lam, phase = params
    arg = 2.0 * np.pi * (X @ dirs.T) / lam + phase
    return 128.0 + 100.0 * np.sin(arg)


def rgb_view(rgb_cam, prims, params, chunk=1 << 19, device=None):
    dw, _ = pixel_rays(rgb_cam)
    d = dw.reshape(-1, 3)
    img = np.zeros((len(d), 3))
    if device is not None:
        chunk = len(d)
    for s in range(0, len(d), chunk):
        dd = d[s:s + chunk]
        t = raycast(prims, rgb_cam.pos, dd, device)
        hit = np.isfinite(t)
        X = rgb_cam.pos + t[hit, None] * dd[hit]
        col = np.zeros((len(dd), 3))
        col[hit] = procedural_colour(X, params)
        img[s:s + chunk] = col
    return np.clip(np.floor(img + 0.5), 0, 255).astype(np.uint8).reshape(rgb_cam.h, rgb_cam.w, 3)


# --------------------------------------------------------------------------- frames

def f32_box(box):
    """The bounding box as the C ABI receives it (float32 per coordinate),
    as float64 values: the oracle must see the same box the kernels see."""
    return tuple(float(np.float32(v)) for v in box)


def frame_config(name):
    """Named workloads: grid, bbox and capture geometry."""
    if name == "sphere64":
        return {"grid_n": (64, 64, 64), "bbox": (-1.2, -1.2, -1.2, 1.2, 1.2, 1.2)}
    if name.startswith("human"):
        n = int(name[len("human"):] or 256)
        return {"grid_n": (n, n, n), "bbox": (-1.0, -0.05, -1.0, 1.0, 1.95, 1.0),
                "K": 4, "ring": 2.5, "height": 1.2}
    raise ValueError(name)


def human_frame(seed=0, K=4, ring=2.5, height=1.2, depth_wh=(512, 424), fxy=365.0,
                rgb_wh=(1920, 1080), rgb_f=1060.0, angle_range=40.0, with_rgb=True,
                noise_coef=0.0012, pixel_stride=1, device=None, yaw_deg=None, pose_seed=None):
    """One synthetic multi-camera frame of the capsule human.

    Returns dict(points [P,3] f32, normals [P,3] f32, weights [P] f32,
    per_camera [(start, count)], views [dict(depth, conf, rgb, K, world_to_cam,
    K_rgb, world_to_rgb)], prims, cams).
    """
    rng = np.random.default_rng(seed)
    # pose_seed: another body pose seen by the same rig (cameras, texture, noise stream of ``seed``)
    prims = human_primitives(seed if pose_seed is None else pose_seed, angle_range, yaw_deg)
    cams = ring_cameras(K, ring, height, (0.0, 0.95, 0.0), depth_wh[0], depth_wh[1], fxy, fxy,
                        phase_deg=float(rng.uniform(0, 360.0 / K)))
    params = texture_params(seed)
    pts, nrms, ws, per_cam, views = [], [], [], [], []
    start = 0
    for cam in cams:
        z = depth_view(cam, prims, rng, noise_coef, device)
        xc, xw = backproject(cam, z)
        nc, valid = organised_normals(xc, z, noise_coef)
        if pixel_stride > 1:
            keep = np.zeros_like(valid)
            keep[::pixel_stride, ::pixel_stride] = True
            valid = valid & keep
        xhat = -xc / np.maximum(np.linalg.norm(xc, axis=-1, keepdims=True), 1e-12)
        w1 = np.maximum(np.sum(xhat * nc, axis=-1), 0.0)
        w2 = box_mean(z > 0, 10)
        W = np.where(valid, w1 * w2, 0.0)
        nw = nc @ cam.R                                 # camera -> world (R^T n)
        P = xw[valid]
        pts.append(P)
        nrms.append(nw[valid])
        ws.append(W[valid])
        per_cam.append((start, len(P)))
        start += len(P)
        view = {"depth": z.astype(np.float32), "conf": W.astype(np.float32),
                "K": cam.K.astype(np.float32), "world_to_cam": cam.world_to_cam.astype(np.float32)}
        if with_rgb:
            rc = rgb_companion(cam, rgb_wh[0], rgb_wh[1], rgb_f, rgb_f)
            view["rgb"] = rgb_view(rc, prims, params, device=device)
            view["K_rgb"] = rc.K.astype(np.float32)
            view["world_to_rgb"] = rc.world_to_cam.astype(np.float32)
        views.append(view)
    return {
        "points": np.concatenate(pts).astype(np.float32),
        "normals": np.concatenate(nrms).astype(np.float32),
        "weights": np.concatenate(ws).astype(np.float32),
        "per_camera": per_cam,
        "views": views,
        "prims": prims,
        "cams": cams,
        "texture_params": params,
    }
