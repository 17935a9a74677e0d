"""Own discrete Fourier transforms for the oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Section III-B of the paper transforms each component of the gradient field
with a 3D FFT and inverts the filtered spectrum with an inverse 3D FFT; it
names no library ("very fast FFT implementations").  The oracle uses its
own transform so that it depends on no FFT library:

* ``dft_brute``  the O(N^2) definition X[k] = sum_n x[n] exp(s 2 pi i n k/N),
  used only to pin ``fft`` on small sizes.
* ``fft``        a mixed-radix (4, 2, 3, 5) Stockham autosort transform,
  derived as follows.  Let N = p_1 ... p_t, L_q = p_1 ... p_q, r_q = N/L_q.
  Y_q[s, k] holds, for each residue s < r_q, the length-L_q DFT of the
  subsequence x[s + r_q n].  Splitting n = p n' + a and k = k' + L_{q-1} b
  gives
      Y_q[s, k' + L_{q-1} b] = sum_a W_p^{ab} W_{L_q}^{a k'} Y_{q-1}[s + r_q a, k'],
  starting from Y_0[s, 0] = x[s] and ending with Y_t[0, k] = X[k].  Each
  stage is one twiddle multiply and one p-point DFT (a p x p matrix product).
Sign convention: forward uses exp(-2 pi i nk/N); the inverse uses
exp(+2 pi i nk/N) and divides by N.
"""

import numpy as np

_RADICES = (4, 2, 3, 5)


def factorize(n):
    """Factor n into the radices 4, 2, 3, 5 (4 first).  Raises for other primes."""
    n = int(n)
    if n < 1:
        raise ValueError("transform length must be positive")
    out = []
    m = n
    for p in _RADICES:
        while m % p == 0:
            out.append(p)
            m //= p
    if m != 1:
        raise ValueError(f"length {n} has a prime factor outside (2, 3, 5)")
    return out


def _unit_root(num, den, sign):
    """exp(sign * 2 pi i * num / den) with num reduced mod den first (float64)."""
    num = np.mod(num, den)
    return np.exp(sign * 2j * np.pi * (num / den))


def dft_brute(x, axis=-1, inverse=False):
    """O(N^2) DFT along ``axis`` straight from the definition (pins ``fft``)."""
    x = np.asarray(x, dtype=np.complex128)
    x = np.moveaxis(x, axis, -1)
    n = x.shape[-1]
    sign = 1.0 if inverse else -1.0
    idx = np.arange(n)
    mat = _unit_root(np.outer(idx, idx), n, sign)          # mat[k, n]
    out = x @ mat.T
    if inverse:
        out = out / n
    return np.moveaxis(out, -1, axis)


def fft(x, axis=-1, inverse=False):
    """Mixed-radix Stockham FFT along ``axis`` (float64 complex)."""
    x = np.asarray(x, dtype=np.complex128)
    x = np.moveaxis(x, axis, -1)
    shape = x.shape
    n = shape[-1]
    sign = 1.0 if inverse else -1.0
    batch = int(np.prod(shape[:-1], dtype=np.int64))
    y = x.reshape(batch, n, 1)                 # Y_0[s, k]: r_0 = n residues, L_0 = 1
    l_prev = 1
    for p in factorize(n):
        l_cur = l_prev * p
        r_cur = n // l_cur
        # Y_{q-1}[s + r_cur a, k'] viewed as [a, s, k']
        y4 = y.reshape(batch, p, r_cur, l_prev)
        a = np.arange(p).reshape(p, 1)
        kp = np.arange(l_prev).reshape(1, l_prev)
        tw = _unit_root(a * kp, l_cur, sign)              # W_{L_q}^{a k'}
        y4 = y4 * tw[None, :, None, :]
        ab = np.arange(p)
        wp = _unit_root(np.outer(ab, ab), p, sign)        # W_p^{ab}, [b, a]
        z = np.einsum("ba,xask->xsbk", wp, y4)            # [batch, s, b, k']
        y = z.reshape(batch, r_cur, l_cur)                # index k' + L_{q-1} b
        l_prev = l_cur
    out = y.reshape(shape)
    if inverse:
        out = out / n
    return np.moveaxis(out, -1, axis)


def fft3(x, inverse=False):
    """3D transform of an array indexed [z, y, x] (all three axes)."""
    out = np.asarray(x, dtype=np.complex128)
    for ax in (2, 1, 0):
        out = fft(out, axis=ax, inverse=inverse)
    return out
