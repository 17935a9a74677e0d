"""The point ingest decides floor(t) and the nearest node from t =
(X - b_min)/h - 1/2 without float64 arithmetic: X - b_min as an exact sum of
two floats, times 1/h held as a float pair, and a fall-back to float64 only
when the fraction lies within 1e-6 of 0, 1/2 or 1.  Restated here in float32
step by step (fmaf emulated exactly) and checked, on random points and on
points placed next to node planes, against the float64 definition: every
decision taken without the fall-back must agree."""

import numpy as np

f32 = np.float32


def _fma(a, b, c):
    # a*b is exact in float64 for float32 a, b; one rounding of the sum to float32
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def _node_t_pair(x, bmin, ih, ih_lo):
    s = f32(x - bmin)
    bb = f32(s - x)
    e = f32(f32(x - f32(s - bb)) + f32(-bmin - bb))
    p = f32(s * ih)
    tl = f32(_fma(s, ih, -p) + _fma(s, ih_lo, f32(e * ih)))
    th = f32(p - f32(0.5))
    if not abs(th) < f32(8388608.0):
        return None
    fl = np.floor(th)
    r = f32(f32(th - fl) + tl)
    fi = int(fl)
    band = f32(1e-6)
    if abs(r) < band or abs(f32(r - f32(1.0))) < band or abs(f32(r - f32(0.5))) < band:
        return None
    if r < 0:
        r = f32(r + f32(1.0))
        fi -= 1
    elif r > 1:
        r = f32(r - f32(1.0))
        fi += 1
    return fi, bool(r > 0.5)


def test_float_pair_decisions_equal_float64():
    rng = np.random.default_rng(3)
    misses = fallbacks = random_fallbacks = total = 0
    for n, (lo, hi) in ((256, (-1.0, 1.0)), (384, (-0.05, 1.95)), (96, (-1.2, 1.2))):
        bmin = f32(lo)
        h = (np.float64(f32(hi)) - np.float64(bmin)) / n
        inv_h = 1.0 / h
        ih = f32(inv_h)
        ih_lo = f32(inv_h - np.float64(ih))
        q = rng.integers(1, n - 2, 20000)
        # random positions, and positions within a few ulps of node planes and midpoints
        xs = [lo + (hi - lo) * rng.random(20000)]
        for off in (0.0, 0.5):
            base = np.float64(bmin) + (q + 0.5 + off) * h
            xs.append(base + rng.integers(-3, 4, q.size) * np.spacing(np.float32(base)).astype(np.float64))
        for j, x in enumerate(np.concatenate(xs).astype(np.float32)):
            t = (np.float64(x) - np.float64(bmin)) / h - 0.5
            got = _node_t_pair(x, bmin, ih, ih_lo)
            total += 1
            if got is None:
                fallbacks += 1
                random_fallbacks += j < 20000
                continue
            fl, up = got
            if fl != int(np.floor(t)) or up != bool(t - np.floor(t) > 0.5):
                misses += 1
    assert misses == 0
    assert random_fallbacks <= 3             # random points almost never need float64
    assert 0 < fallbacks < 0.5 * total       # points within ~1e-6 of a plane do; most near-plane points do not
