"""Spectral integration of the gradient field into the indicator A (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. III-B: each component V_c is transformed with a 3D FFT, the integration
filter F(w) = (1/|w|^2) [j w_x, j w_y, j w_z] is applied by multiplication,
and A is the inverse 3D FFT of the filtered field summed over the three
components.  By linearity the sum of the three inverse transforms equals one
inverse transform of the summed spectrum, which is what is computed here:

  A^(k) = j (w_x V^_x + w_y V^_y + w_z V^_z) / |w|^2,    A = IDFT_3(A^)

Readings (``oracle.conventions``): w_c = 2 pi k_c / (n_c h_c) with signed
k_c; the numerator w_c is 0 at the Nyquist index k_c = n_c/2 while the
denominator uses |k_c| = n_c/2; A^(0) = 0.  The transform is the oracle's own
complex FFT of the real field; the imaginary part of the result is checked
to be at rounding level and dropped.
"""

import numpy as np

from . import conventions as cv
from . import fft as offt


def omega_axis(n, h):
    """Return (numerator w, denominator w) for one axis of length n, spacing h."""
    k = np.arange(n)
    ks = np.where(k < n // 2, k, k - n).astype(np.float64)   # signed, Nyquist -> -n/2
    den = 2.0 * np.pi * ks / (n * h)
    num = den.copy()
    if n % 2 == 0:
        num[n // 2] = 0.0
    return num, den


def filter_spectrum(Vhat, grid_n, bbox):
    """Apply F(w) and sum the components: Vhat [3, nz, ny, nx] -> A^ [nz, ny, nx]."""
    nx, ny, nz = (int(v) for v in grid_n)
    h = cv.voxel_size(grid_n, bbox)
    nwx, dwx = omega_axis(nx, h[0])
    nwy, dwy = omega_axis(ny, h[1])
    nwz, dwz = omega_axis(nz, h[2])
    num = (nwx[None, None, :] * Vhat[0]
           + nwy[None, :, None] * Vhat[1]
           + nwz[:, None, None] * Vhat[2])
    den = dwx[None, None, :] ** 2 + dwy[None, :, None] ** 2 + dwz[:, None, None] ** 2
    out = np.zeros_like(num)
    nz_mask = den > 0
    out[nz_mask] = 1j * num[nz_mask] / den[nz_mask]
    return out


def integrate(V, grid_n, bbox, return_spectrum=False):
    """V [3, nz, ny, nx] (real) -> A [nz, ny, nx] (real, float64)."""
    Vhat = np.stack([offt.fft3(V[c]) for c in range(3)])
    Ahat = filter_spectrum(Vhat, grid_n, bbox)
    Ac = offt.fft3(Ahat, inverse=True)
    A = Ac.real.copy()
    # A is of order |V| h; the imaginary part must be at rounding level of that
    h = cv.voxel_size(grid_n, bbox)
    scale = max(float(np.max(np.abs(A))), float(np.max(np.abs(V))) * max(h), 1e-300)
    if float(np.max(np.abs(Ac.imag))) > 1e-9 * scale:
        raise AssertionError("inverse transform is not real: filter lost Hermitian symmetry")
    if return_spectrum:
        return A, Ahat
    return A
