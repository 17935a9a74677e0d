"""Named readings of points the paper leaves silent (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Every constant here is one reading of Section III-B/III-C of the paper; the
CUDA library states the same readings independently in its own source.

* Grid nodes are cell-centred: p(q) = b_min + (q + 1/2) h, h = extent / n
  (Sec. III-B: "grid q ... inside the bounding box").
* g(x; s) = s^-1 exp(-x^2 / s^2), taken literally (eq. (1), (2)).
* sigma1 = half the voxel diagonal, sigma2^2 = 3/2 sigma1^2 (Sec. III-B).
* Stencil: with t = (X - b_min)/h - 1/2, nodes floor(t)-1 .. floor(t)+2 on
  every axis ("the 4^3 voxels around each input point", Sec. III-B).
* A point is accepted iff 1 <= t < n-2 on every axis, i.e. its whole stencil
  lies inside the grid; other points are dropped and counted.
* Simple splat: the nearest node floor(t + 1/2), count-normalised, W ignored
  (Sec. III-B, "simplest nonweighted version").
* DFT: forward kernel exp(-2 pi i k.n / N), inverse carries 1/M.
* omega_c = 2 pi k_c / (n_c h_c) with signed k_c in [-n_c/2, n_c/2); the
  numerator omega_c is 0 at the Nyquist index k_c = n_c/2, the denominator
  uses |k_c| = n_c/2 there; A^(0) = 0.
* Level: unweighted mean over accepted points of trilinear A (Sec. III-B).
* Marching cubes: corner bit = 1 iff A >= L compared in float64.
"""

SIGMA2_RATIO2 = 1.5          # sigma2^2 / sigma1^2, Sec. III-B ("sigma2^2 = 3/2 sigma1^2")

# Raw reconstruction (Sec. III-A).  The paper triangulates each depth map
# (the organised-point method of its ref. [13]) and skips triangles across
# depth discontinuities without giving the threshold; the reading here: a
# triangle is kept iff all three pixels are foreground and the largest depth
# difference among its corners is <= TSDC_STEP + 3 sigma(z_max) with the
# depth noise sigma(z) = TSDC_NOISE z^2 (metres).  W2 is the mean of the
# binary silhouette over a (2 W2_RADIUS + 1)^2 window, zero outside the image.
TSDC_STEP = 0.03
TSDC_NOISE = 0.0012
W2_RADIUS = 10
STENCIL = 4                  # 4^3 support, Sec. III-B
STENCIL_LO = 1               # nodes floor(t)-1 .. floor(t)+2
SPLAT_WEIGHTED = 0
SPLAT_SIMPLE = 1


def voxel_size(grid_n, bbox):
    """h_c = (b_max,c - b_min,c) / n_c for c = x, y, z (cell-centred grid)."""
    return tuple((float(bbox[3 + c]) - float(bbox[c])) / int(grid_n[c]) for c in range(3))


def sigmas(grid_n, bbox, sigma1_scale=1.0, sigma2_ratio2=SIGMA2_RATIO2):
    """sigma1 = scale * half voxel diagonal; sigma2 = sqrt(ratio2) * sigma1 (Sec. III-B)."""
    h = voxel_size(grid_n, bbox)
    s1 = sigma1_scale * 0.5 * (h[0] ** 2 + h[1] ** 2 + h[2] ** 2) ** 0.5
    s2 = (sigma2_ratio2 ** 0.5) * s1
    return s1, s2
