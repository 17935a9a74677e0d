"""Objective evaluation of a reconstruction against sensor views (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. III-E compares the mesh, rendered into each of the K + K' views, with
what the sensor captured there:

* eq. (3)  VRE  V_k = |S_r xor S_g| / |S_r or S_g| on the silhouettes
  (S_r: drawn pixels of the rendered depth, S_g: foreground of the sensor
  depth);
* eq. (4)  the symmetric 2D Hausdorff distance H_k between the silhouettes,
  in pixels;
* eq. (5)  CP-RMSE: the root mean square, over the points back-projected
  from the sensor's foreground depth, of the distance to the closest point
  back-projected from the rendered depth;
* eq. (6)(7) WMS3IM: SSIM terms l, c, s per pixel over a window N(u),
  averaged over the rendered silhouette with weights w(u) = |N(u) and S_r|,
  at J = 3 scales, combined as prod_j l_j^a_j c_j^b_j s_j^g_j.

Readings:

* back-projection uses the rasteriser's pixel ray (``oracle.render``):
  X = z (dx, dy, 1) in camera coordinates (the distances do not depend on
  the camera pose);
* empty sets: VRE = 0 and H = 0 when both silhouettes are empty; H = inf
  when only one is; CP-RMSE = nan without sensor points, inf without
  rendered points;
* SSIM works on the luma Y = 0.299 R + 0.587 G + 0.114 B of the 8-bit
  images; N(u) is the 11 x 11 window around u with the Gaussian weights
  exp(-t^2 / (2 * 1.5^2)) per axis, cut at the image border and
  renormalised to sum 1 there; C1 = (0.01 * 255)^2, C2 = (0.03 * 255)^2,
  C3 = C2 / 2 (the constants of the SSIM index the paper cites);
* the structure term is s = (sigma_XY + C3) / (sigma_X sigma_Y + C3): the
  factor 2 printed in its numerator would give identical images s > 1,
  against the cited index;
* sigma_X = sqrt(max(E[X^2] - mu_X^2, 0)); w(u) counts the silhouette
  pixels of the same (cut) 11 x 11 window;
* scale j + 1 is the 2 x 2 block mean of scale j (size floor(n / 2)) and its
  silhouette the 2 x 2 block AND;
* a weighted mean that is <= 0 contributes 0 to the product (a negative
  base has no real power); without silhouette pixels at some scale all
  terms and WMS3IM are nan.
"""

import numpy as np

from oracle.render import pixel_ray

SSIM_RADIUS = 5
SSIM_SIGMA = 1.5
SSIM_C1 = (0.01 * 255.0) ** 2
SSIM_C2 = (0.03 * 255.0) ** 2
SSIM_C3 = SSIM_C2 / 2.0
# Sec. III-E3: exponents of the J = 3 scales (luminance, contrast, structure)
WMS3IM_ALPHA = (0.0, 0.0, 0.1333)
WMS3IM_BETA = (0.0448, 0.3001, 0.1333)
WMS3IM_GAMMA = (0.0448, 0.3001, 0.1333)
LUMA = (0.299, 0.587, 0.114)


def silhouettes(rendered_depth, sensor_depth):
    return np.asarray(rendered_depth) > 0, np.asarray(sensor_depth) > 0


def vre(rendered_depth, sensor_depth):
    """eq. (3): (V_k, |S_r xor S_g|, |S_r or S_g|, |S_r|, |S_g|)."""
    r, g = silhouettes(rendered_depth, sensor_depth)
    x = int(np.count_nonzero(r ^ g))
    o = int(np.count_nonzero(r | g))
    return (x / o if o else 0.0), x, o, int(r.sum()), int(g.sum())


def _directed_sq(p, q, chunk=256):
    """max over p of the squared distance to the nearest of q (brute force)."""
    worst = 0
    for s in range(0, len(p), chunk):
        d = p[s:s + chunk, None, :] - q[None, :, :]
        worst = max(worst, int((d * d).sum(-1).min(axis=1).max()))
    return worst


def hausdorff(rendered_depth, sensor_depth):
    """eq. (4): symmetric 2D Hausdorff distance between the silhouettes, pixels."""
    r, g = silhouettes(rendered_depth, sensor_depth)
    pr = np.argwhere(r).astype(np.int64)
    pg = np.argwhere(g).astype(np.int64)
    if len(pr) == 0 or len(pg) == 0:
        return 0.0 if len(pr) == len(pg) else float("inf")
    return float(np.sqrt(max(_directed_sq(pr, pg), _directed_sq(pg, pr))))


def backproject(K, depth):
    """Camera-space points [n, 3] of the pixels with depth > 0 (row-major order)."""
    depth = np.asarray(depth)
    jj, ii = np.nonzero(depth > 0)
    dx, dy = pixel_ray(K, ii.astype(np.float64), jj.astype(np.float64))
    z = depth[jj, ii].astype(np.float64)
    return np.stack([z * dx, z * dy, z], axis=1)


def closest_sq(P, Q, chunk=128):
    """Squared distance from each point of P to the closest point of Q (brute force)."""
    out = np.empty(len(P))
    for s in range(0, len(P), chunk):
        d = P[s:s + chunk, None, :] - Q[None, :, :]
        out[s:s + chunk] = (d * d).sum(-1).min(axis=1)
    return out


def cp_rmse(K, rendered_depth, sensor_depth):
    """eq. (5): (CP-RMSE_k, I_k sensor points, J_k rendered points)."""
    Xg = backproject(K, sensor_depth)
    Xr = backproject(K, rendered_depth)
    if len(Xg) == 0:
        return float("nan"), 0, len(Xr)
    if len(Xr) == 0:
        return float("inf"), len(Xg), 0
    return float(np.sqrt(closest_sq(Xg, Xr).mean())), len(Xg), len(Xr)


def luma(rgb):
    rgb = np.asarray(rgb, dtype=np.float64)
    return LUMA[0] * rgb[..., 0] + LUMA[1] * rgb[..., 1] + LUMA[2] * rgb[..., 2]


def gaussian_taps():
    t = np.arange(-SSIM_RADIUS, SSIM_RADIUS + 1, dtype=np.float64)
    return np.exp(-t * t / (2.0 * SSIM_SIGMA * SSIM_SIGMA))


def _overlap(n, d):
    """(destination, source) slices of the pixels i with 0 <= i + d < n
    (empty when |d| >= n)."""
    lo, hi = max(0, -d), min(n, n - d)
    if hi <= lo:
        return slice(0, 0), slice(0, 0)
    return slice(lo, hi), slice(lo + d, hi + d)


def window_mean(img, taps):
    """Weighted mean over the (2R+1)^2 window around every pixel, the window
    cut at the border and its weights renormalised to 1."""
    h, w = img.shape
    R = (len(taps) - 1) // 2
    num = np.zeros((h, w))
    den = np.zeros((h, w))
    for dy in range(-R, R + 1):
        for dx in range(-R, R + 1):
            wt = taps[dy + R] * taps[dx + R]
            ys, yd = _overlap(h, dy)
            xs, xd = _overlap(w, dx)
            num[ys, xs] += wt * img[yd, xd]
            den[ys, xs] += wt
    return num / den


def window_count(mask, R=SSIM_RADIUS):
    """w(u): silhouette pixels in the (2R+1)^2 window around u, cut at the border."""
    h, w = mask.shape
    m = mask.astype(np.int64)
    out = np.zeros((h, w), np.int64)
    for dy in range(-R, R + 1):
        for dx in range(-R, R + 1):
            ys, yd = _overlap(h, dy)
            xs, xd = _overlap(w, dx)
            out[ys, xs] += m[yd, xd]
    return out


def ssim_maps(X, Y):
    """Per-pixel luminance, contrast and structure terms, eq. (6)."""
    g = gaussian_taps()
    mx = window_mean(X, g)
    my = window_mean(Y, g)
    vx = np.maximum(window_mean(X * X, g) - mx * mx, 0.0)
    vy = np.maximum(window_mean(Y * Y, g) - my * my, 0.0)
    cxy = window_mean(X * Y, g) - mx * my
    sx = np.sqrt(vx)
    sy = np.sqrt(vy)
    l = (2.0 * mx * my + SSIM_C1) / (mx * mx + my * my + SSIM_C1)
    c = (2.0 * sx * sy + SSIM_C2) / (vx + vy + SSIM_C2)
    s = (cxy + SSIM_C3) / (sx * sy + SSIM_C3)
    return l, c, s


def downsample(X, S):
    """Next scale: 2 x 2 block mean of the image, 2 x 2 block AND of the silhouette."""
    h, w = X.shape[0] // 2, X.shape[1] // 2
    Xc = X[:2 * h, :2 * w]
    Sc = S[:2 * h, :2 * w]
    Xn = 0.25 * (Xc[0::2, 0::2] + Xc[0::2, 1::2] + Xc[1::2, 0::2] + Xc[1::2, 1::2])
    Sn = Sc[0::2, 0::2] & Sc[0::2, 1::2] & Sc[1::2, 0::2] & Sc[1::2, 1::2]
    return Xn, Sn


def wms3im(rendered_depth, rendered_rgb, sensor_rgb, scales=3):
    """eq. (6)(7): (WMS3IM, l [J], c [J], s [J]) over the rendered silhouette."""
    X = luma(rendered_rgb)
    Y = luma(sensor_rgb)
    S = np.asarray(rendered_depth) > 0
    L, C, Sg = [], [], []
    for j in range(scales):
        if j:
            X, S1 = downsample(X, S)
            Y, _ = downsample(Y, S)
            S = S1
        wts = window_count(S).astype(np.float64) * S
        tot = wts.sum()
        if tot == 0:
            nan = [float("nan")] * scales
            return float("nan"), nan, nan, nan
        l, c, s = ssim_maps(X, Y)
        L.append(float((l * wts).sum() / tot))
        C.append(float((c * wts).sum() / tot))
        Sg.append(float((s * wts).sum() / tot))
    out = 1.0
    for j in range(scales):
        for val, e in ((L[j], WMS3IM_ALPHA[j]), (C[j], WMS3IM_BETA[j]), (Sg[j], WMS3IM_GAMMA[j])):
            if e != 0.0:
                out *= max(val, 0.0) ** e
    return out, L, C, Sg
