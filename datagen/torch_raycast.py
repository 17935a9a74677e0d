"""Ray casting of the capsule/ellipsoid body with torch (input generation only).

The same closed-form ray-capsule and ray-ellipsoid intersections as
``datagen.scenes`` (float64), evaluated with torch so that large RGB views
and many sessions can be generated on a GPU in the benchmark.  The numpy
version in ``scenes`` remains the one the tests use.
"""

import numpy as np


def _sphere(o, d, c, r, torch):
    oc = o - c
    b = (oc * d).sum(-1)
    cc = (oc * oc).sum(-1) - r * r
    disc = b * b - cc
    t = -b - torch.sqrt(torch.clamp(disc, min=0.0))
    return torch.where(disc >= 0, t, torch.full_like(t, float("inf")))


def _capsule(o, d, cap, torch):
    a = torch.as_tensor(cap.a, dtype=d.dtype, device=d.device)
    b = torch.as_tensor(cap.b, dtype=d.dtype, device=d.device)
    ba = b - a
    L = torch.sqrt((ba * ba).sum())
    u = ba / L
    oa = o - a
    du = d @ u
    ou = oa @ u
    dp = d - du[:, None] * u
    op = oa - ou[..., None] * u
    A = (dp * dp).sum(-1)
    B = (dp * op).sum(-1)
    C = (op * op).sum(-1) - cap.r ** 2
    disc = B * B - A * C
    t = (-B - torch.sqrt(torch.clamp(disc, min=0.0))) / torch.clamp(A, min=1e-300)
    y = ou + t * du
    inf = torch.full_like(t, float("inf"))
    tc = torch.where((disc >= 0) & (A > 1e-12) & (y >= 0) & (y <= L), t, inf)
    t1 = _sphere(o, d, a, cap.r, torch)
    t2 = _sphere(o, d, b, cap.r, torch)
    t = torch.minimum(tc, torch.minimum(t1, t2))
    return torch.where(t > 1e-6, t, inf)


def _ellipsoid(o, d, el, torch):
    M = torch.as_tensor(el.R / el.radii[:, None], dtype=d.dtype, device=d.device)
    c = torch.as_tensor(el.c, dtype=d.dtype, device=d.device)
    op = (o - c) @ M.T
    dp = d @ M.T
    a = (dp * dp).sum(-1)
    b = (op * dp).sum(-1)
    cc = (op * op).sum(-1) - 1.0
    disc = b * b - a * cc
    t = (-b - torch.sqrt(torch.clamp(disc, min=0.0))) / a
    return torch.where((disc >= 0) & (t > 1e-6), t, torch.full_like(t, float("inf")))


def raycast_torch(prims, origin, dirs, device):
    """Nearest hit distance along unit rays (numpy in, numpy out)."""
    import torch
    from .scenes import Capsule
    d = torch.as_tensor(np.asarray(dirs, dtype=np.float64), device=device)
    o = torch.as_tensor(np.asarray(origin, dtype=np.float64), device=device)
    best = torch.full((d.shape[0],), float("inf"), dtype=torch.float64, device=device)
    for p in prims:
        t = _capsule(o, d, p, torch) if isinstance(p, Capsule) else _ellipsoid(o, d, p, torch)
        best = torch.minimum(best, t)
    return best.cpu().numpy()
