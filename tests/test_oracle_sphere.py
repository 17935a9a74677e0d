"""End-to-end oracle pins on the analytic sphere (64^3 over [-1.2, 1.2]^3), no GPU.

For a locally flat, uniformly sampled surface, eq. (1)(2) give a gradient
field V(s) = sqrt(2/3) exp(-s^2 / (3 sigma1^2)) N across the surface (s the
signed distance), so the indicator jumps by dA = sqrt(2 pi) sigma1 and its
level set at the mean of A on the samples is the sphere itself.
"""

import numpy as np
import pytest

from datagen import frame_config, sphere_points
from oracle import conventions as cv
from oracle import pipeline
from tests.test_oracle_mc import _edge_check


@pytest.fixture(scope="module")
def sphere_run():
    cfg = frame_config("sphere64")
    P, N, W = sphere_points(20000, 0.005, seed=0)
    return cfg, P, pipeline.reconstruct(P, N, W, cfg["grid_n"], cfg["bbox"])


def test_indicator_jump_matches_flat_surface_closed_form(sphere_run):
    cfg, _, r = sphere_run
    A = r["A"]
    s1, _ = cv.sigmas(cfg["grid_n"], cfg["bbox"])
    inside = A[28:36, 28:36, 28:36].mean()
    outside = np.concatenate([A[:3].ravel(), A[-3:].ravel()]).mean()
    assert abs((inside - outside) / (np.sqrt(2 * np.pi) * s1) - 1.0) < 0.10
    assert inside > r["L"] > outside


def test_radial_profile_is_erfc_like(sphere_run):
    cfg, _, r = sphere_run
    A = r["A"]
    n = 64
    h = 2.4 / n
    c = (np.arange(n) + 0.5) * h - 1.2
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    rad = np.sqrt(x * x + y * y + z * z)
    prof = [A[(rad > a) & (rad < a + h)].mean() for a in np.arange(0.7, 1.3, h)]
    assert np.all(np.diff(prof) < 1e-3)          # decreasing across the surface
    mid = 0.5 * (max(prof) + min(prof))
    cross = np.arange(0.7, 1.3, h)[np.argmin(np.abs(np.array(prof) - mid))] + 0.5 * h
    assert abs(cross - 1.0) < 1.5 * h


def test_sphere_mesh_radius_and_topology(sphere_run):
    cfg, _, r = sphere_run
    m = r["mesh"]
    h = 2.4 / 64
    rad = np.linalg.norm(m["vertices"], axis=1)
    assert abs(rad.mean() - 1.0) <= 0.25 * h
    assert np.max(np.abs(rad - 1.0)) <= h
    w, o, chi, comps = _edge_check(m["tris"])
    assert w and o and chi == 2 and comps == 1
    assert np.all(np.einsum("ij,ij->i", m["normals"], m["vertices"]) > 0)


def test_simple_mode_also_closes(sphere_run):
    cfg, P, _ = sphere_run
    _, N, W = sphere_points(20000, 0.005, seed=0)
    r = pipeline.reconstruct(P, N, W, cfg["grid_n"], cfg["bbox"], mode=cv.SPLAT_SIMPLE)
    rad = np.linalg.norm(r["mesh"]["vertices"], axis=1)
    assert abs(rad.mean() - 1.0) <= 0.5 * 2.4 / 64
    w, o, chi, _ = _edge_check(r["mesh"]["tris"])
    assert w and o and chi == 2
