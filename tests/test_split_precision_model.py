"""Error model of the split-precision DFT stages (BF16x3 / FP16x3): a batch
of complex vectors times the real 2R x 2R DFT matrix, both operands split
into 16-bit hi/lo parts, three products (lo.hi + hi.lo + hi.hi) accumulated
in float32.  Emulated here with exact 16-bit rounding and float32 sums, and
compared with the float64 product: the relative error of one stage stays
within 2 u^2 (u = 2^-9 for bf16, 2^-11 for fp16) plus float32
accumulation, the per-stage figure behind the tests' error bars (twelve
stages, two per axis and direction)."""

import numpy as np


def _bf16(x):
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def _fp16(x):
    return np.asarray(x, np.float32).astype(np.float16).astype(np.float32)


def _split(x, rnd):
    hi = rnd(x)
    lo = rnd((x - hi).astype(np.float32))
    return hi, lo


def _dft_matrix(R):
    """Real 2R x 2R matrix of the length-R forward DFT on (re, im) interleaved rows."""
    k = np.arange(R)
    W = np.exp(-2j * np.pi * np.outer(k, k) / R)
    D = np.zeros((2 * R, 2 * R))
    D[0::2, 0::2] = W.real.T
    D[1::2, 0::2] = -W.imag.T
    D[0::2, 1::2] = W.imag.T
    D[1::2, 1::2] = W.real.T
    return D


def _stage(X, D, rnd, scale):
    X = X.astype(np.float32)
    s = np.ones((X.shape[0], 1), np.float32)
    if scale:          # fp16: each row scaled by a power of two into [1/2, 1) first (exact)
        m = np.max(np.abs(X), axis=1, keepdims=True)
        e = np.ceil(np.log2(np.maximum(m, 1e-30))).astype(np.int32)
        s = np.ldexp(np.float32(1.0), e).astype(np.float32)
        X = (X / s).astype(np.float32)
    xh, xl = _split(X, rnd)
    dh, dl = _split(D.astype(np.float32), rnd)
    # every 16-bit x 16-bit product is exact in float32; the sums are float32
    y = np.zeros((X.shape[0], D.shape[1]), np.float32)
    for a, b in ((xl, dh), (xh, dl), (xh, dh)):
        for k in range(D.shape[0]):
            y = (y + (a[:, k:k + 1] * b[k:k + 1, :]).astype(np.float32)).astype(np.float32)
    return (y * s).astype(np.float64)


def test_one_split_stage_stays_within_the_model():
    rng = np.random.default_rng(5)
    for R in (8, 16, 32):
        D = _dft_matrix(R)
        X = rng.standard_normal((256, 2 * R)).astype(np.float32) * np.float32(3.0)
        exact = X.astype(np.float64) @ D
        # the matrix is the DFT: it reproduces numpy's transform
        z = X[:, 0::2].astype(np.float64) + 1j * X[:, 1::2]
        fz = np.fft.fft(z, axis=1)
        assert np.allclose(exact[:, 0::2] + 1j * exact[:, 1::2], fz, atol=1e-9)
        scale_ref = np.linalg.norm(exact)
        for rnd, u, scale in ((_bf16, 2.0 ** -9, False), (_fp16, 2.0 ** -11, True)):
            err = np.linalg.norm(_stage(X, D, rnd, scale) - exact) / scale_ref
            acc = 2 * np.sqrt(2 * R) * 2.0 ** -24      # float32 accumulation over 3 x 2R terms
            assert 0.1 * u * u < err <= 2 * u * u + acc, (R, u, err)   # measured: 0.6-0.9 u^2 (bf16)
            # the lo.lo term is what the three products leave out: dropping
            # a second one (hi.hi only) is far worse
            xh = rnd(X if not scale else X)
            assert np.linalg.norm(xh.astype(np.float64) @ rnd(D.astype(np.float32)) - exact) / scale_ref > 10 * err
