"""The raw reconstruction (Sec. III-A) keeps or drops each triangle of the
organised depth-map triangulation and orients its normal in float32, and
hands a pixel to float64 when a decision falls inside a guard band (the
depth-step threshold within 1e-5 relative, a nearly degenerate triangle, a
normal nearly perpendicular to the centroid ray).  Restated here step by step
in float32 (edges from exact depth differences, as the kernel forms them)
and in float64 (the plain definition), over every triangle of synthetic
human depth maps: wherever float32 decides, it decides as float64 does."""

import numpy as np

from datagen import human_frame
from oracle import conventions as cv

f32 = np.float32


def _triangles(h, w):
    """(u0, v0) and corner offsets of the two triangle families of every quad."""
    vv, uu = np.mgrid[0:h - 1, 0:w - 1]
    fams = (((0, 0), (1, 0), (0, 1)), ((1, 0), (1, 1), (0, 1)))
    return uu.ravel(), vv.ravel(), fams


def _decide64(D, K, u0, v0, cn, step, noise):
    fx, fy, cx, cy = (np.float64(f32(K[0, 0])), np.float64(f32(K[1, 1])), np.float64(f32(K[0, 2])),
                      np.float64(f32(K[1, 2])))
    P, Z = [], []
    for du, dv in cn:
        u, v = u0 + du, v0 + dv
        z = D[v, u].astype(np.float64)
        Z.append(z)
        P.append(np.stack([(u - cx) / fx * z, (v - cy) / fy * z, z], 1))
    Z = np.stack(Z, 1)
    fg = (Z > 0).all(1)
    zmax = Z.max(1)
    dz = np.maximum(np.maximum(abs(Z[:, 0] - Z[:, 1]), abs(Z[:, 1] - Z[:, 2])), abs(Z[:, 0] - Z[:, 2]))
    thr = step + 3.0 * noise * zmax * zmax
    n = np.cross(P[1] - P[0], P[2] - P[0])
    ln = np.linalg.norm(n, axis=1)
    keep = fg & (dz <= thr) & (ln > 0)
    cen = (P[0] + P[1] + P[2]) / 3.0
    flip = (n * cen).sum(1) > 0
    return keep, flip


def _decide32(D, K, u0, v0, cn, step, noise):
    """-1 undecided, 0 dropped, 1 kept; and the orientation flip where kept."""
    fx, fy, cx, cy = f32(K[0, 0]), f32(K[1, 1]), f32(K[0, 2]), f32(K[1, 2])
    step, noise = f32(step), f32(noise)
    Z = np.stack([D[v0 + dv, u0 + du].astype(f32) for du, dv in cn], 1)
    fg = (Z > 0).all(1)
    zmax = Z.max(1)
    dz = np.maximum(np.maximum(abs(Z[:, 0] - Z[:, 1]), abs(Z[:, 1] - Z[:, 2])), abs(Z[:, 0] - Z[:, 2]))
    thr = (step + ((f32(3.0) * noise) * zmax) * zmax).astype(f32)
    res = np.where(fg, 1, 0)
    und = fg & (abs(dz - thr) <= f32(1e-5) * thr)
    res[fg & ~und & (dz > thr)] = 0
    e = []
    ua, va = (u0 + cn[0][0]).astype(f32), (v0 + cn[0][1]).astype(f32)
    for k in (1, 2):
        du, dv = f32(cn[k][0] - cn[0][0]), f32(cn[k][1] - cn[0][1])
        dd = (Z[:, k] - Z[:, 0]).astype(f32)
        e.append(np.stack([((du * Z[:, k]).astype(f32) + ((ua - cx) * dd).astype(f32)) / fx,
                           ((dv * Z[:, k]).astype(f32) + ((va - cy) * dd).astype(f32)) / fy, dd], 1).astype(f32))
    n = np.cross(e[0], e[1]).astype(f32)
    ln = np.sqrt((n * n).sum(1, dtype=f32)).astype(f32)
    el = (np.sqrt((e[0] * e[0]).sum(1, dtype=f32)) * np.sqrt((e[1] * e[1]).sum(1, dtype=f32))).astype(f32)
    und |= (res == 1) & ~(ln > f32(1e-5) * el)
    cen = np.zeros_like(n)
    for k, (du, dv) in enumerate(cn):
        z = Z[:, k]
        cen[:, 0] += (((u0 + du).astype(f32) - cx) / fx * z).astype(f32)
        cen[:, 1] += (((v0 + dv).astype(f32) - cy) / fy * z).astype(f32)
        cen[:, 2] += z
    dot = (n * cen).sum(1, dtype=f32)
    cl = np.sqrt((cen * cen).sum(1, dtype=f32)).astype(f32)
    und |= (res == 1) & (abs(dot) <= f32(1e-4) * ln * cl)
    res[und] = -1
    return res, dot > 0


def test_float32_triangle_decisions_equal_float64():
    checked = undecided = 0
    for seed in (21, 22):
        fr = human_frame(seed=seed, K=2, with_rgb=False)
        for v in fr["views"]:
            D = v["depth"].astype(np.float32)
            K = v["K"]
            h, w = D.shape
            u0, v0, fams = _triangles(h, w)
            for cn in fams:
                keep, flip = _decide64(D, K, u0, v0, cn, cv.TSDC_STEP, cv.TSDC_NOISE)
                res, flip32 = _decide32(D, K, u0, v0, cn, cv.TSDC_STEP, cv.TSDC_NOISE)
                dec = res >= 0
                assert np.array_equal(res[dec] == 1, keep[dec])
                both = dec & (res == 1)
                assert np.array_equal(flip32[both], flip[both])
                checked += int(both.sum())
                undecided += int((~dec).sum())
    assert checked > 20000 and undecided < 0.01 * checked
