"""Pins for the oracle's spectral integration (Sec. III-B filter jw/|w|^2), no GPU.

Closed form: for a band-limited trigonometric polynomial f on the node grid
(no Nyquist terms), V = -grad f gives A = f - mean(f) to rounding.  This pins
the filter's sign, the units of w, the DC handling and the inverse scaling.
"""

import numpy as np
import pytest

from oracle import conventions as cv
from oracle import spectral


def _trig_field(grid_n, bbox, seed):
    rng = np.random.default_rng(seed)
    nx, ny, nz = grid_n
    h = cv.voxel_size(grid_n, bbox)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    f = np.zeros((nz, ny, nx))
    V = np.zeros((3, nz, ny, nx))
    for _ in range(6):
        k = np.array([rng.integers(-(n // 2) + 1, n // 2) for n in grid_n])
        a = rng.uniform(-1, 1)
        ph = rng.uniform(0, 2 * np.pi)
        arg = 2 * np.pi * (k[0] * x / nx + k[1] * y / ny + k[2] * z / nz) + ph
        f += a * np.cos(arg)
        # d/dx_world of cos(2 pi k_x q_x / n_x + ...) with q_x = (x_w - b)/h - 1/2
        for c, n in enumerate(grid_n):
            V[c] += a * np.sin(arg) * (2 * np.pi * k[c] / (n * h[c]))   # V = -grad f
    return f, V


@pytest.mark.parametrize("grid_n,bbox", [
    ((8, 8, 8), (-1, -1, -1, 1, 1, 1)),
    ((12, 16, 6), (-0.3, 0.1, -2.0, 0.9, 1.7, 0.4)),
    ((16, 32, 16), (0, 0, 0, 1, 2, 1)),
])
def test_closed_form_potential(grid_n, bbox):
    f, V = _trig_field(grid_n, bbox, seed=sum(grid_n))
    A = spectral.integrate(V, grid_n, bbox)
    assert np.max(np.abs(A - (f - f.mean()))) < 1e-12 * max(1.0, np.max(np.abs(f)))


def test_sign_convention_inside_is_larger():
    """Outward normals on a sphere-like blob give A larger inside (grad A ~ -V)."""
    n = 32
    grid = (n, n, n)
    bbox = (-1, -1, -1, 1, 1, 1)
    h = 2.0 / n
    c = (np.arange(n) + 0.5) * h - 1
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt(x * x + y * y + z * z) + 1e-12
    shell = np.exp(-((r - 0.5) / (1.5 * h)) ** 2)
    V = np.stack([shell * x / r, shell * y / r, shell * z / r])
    A = spectral.integrate(V, grid, bbox)
    assert A[n // 2, n // 2, n // 2] > A[0, 0, 0] + 0.5 * np.sqrt(np.pi) * 1.5 * h * 0.5


def test_nyquist_and_dc():
    num, den = spectral.omega_axis(8, 0.25)
    assert num[4] == 0.0 and den[4] != 0.0 and abs(den[4]) == 2 * np.pi * 4 / (8 * 0.25)
    assert num[0] == 0.0 and den[0] == 0.0
    # a field that only lives at Nyquist along x integrates to zero (numerator 0)
    grid = (8, 4, 4)
    x = np.arange(8)
    V = np.zeros((3, 4, 4, 8))
    V[0] = np.cos(np.pi * x)[None, None, :]
    A = spectral.integrate(V, grid, (0, 0, 0, 1, 1, 1))
    assert np.max(np.abs(A)) < 1e-14
    # constant field: all energy at DC -> A = 0
    V = np.ones((3, 4, 4, 8))
    assert np.max(np.abs(spectral.integrate(V, grid, (0, 0, 0, 1, 1, 1)))) < 1e-14


def test_linearity_of_component_sum():
    """One inverse of the summed spectrum equals the sum of three inverses (Sec. III-B)."""
    from oracle import fft as F
    rng = np.random.default_rng(2)
    grid = (8, 12, 6)
    bbox = (0, 0, 0, 1, 1.5, 0.75)
    V = rng.standard_normal((3, 6, 12, 8))
    A = spectral.integrate(V, grid, bbox)
    h = cv.voxel_size(grid, bbox)
    parts = []
    for comp in range(3):
        Vhat = np.zeros((3,) + V.shape[1:], complex)
        Vhat[comp] = F.fft3(V[comp])
        parts.append(F.fft3(spectral.filter_spectrum(Vhat, grid, bbox), inverse=True).real)
    assert np.max(np.abs(A - sum(parts))) < 1e-12
    assert abs(A.mean()) < 1e-14
    assert h[1] == 0.125
