"""Pins for the oracle's Fourier transform (the F-hat of Eq. 2): brute-force DFT from the definition,
numpy.fft as an independent library, and closed forms (delta, plane wave, Parseval)."""
import itertools

import numpy as np
import pytest

import oracle


def brute_dft4(f, sign):
    """O(V^2) 4D DFT straight from the definition, f indexed (t, z, y, x)."""
    nt, nz, ny, nx = f.shape
    out = np.zeros_like(f)
    xs = list(itertools.product(range(nt), range(nz), range(ny), range(nx)))
    for k in xs:
        acc = 0j
        for x in xs:
            ph = sum(k[a] * x[a] / f.shape[a] for a in range(4))
            acc += f[x] * np.exp(sign * 2j * np.pi * ph)
        out[k] = acc
    return out


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 16, 24, 27, 32, 48, 64])
def test_fft1d_brute(N):
    rng = np.random.default_rng(N)
    f = rng.normal(size=N) + 1j * rng.normal(size=N)
    j = np.arange(N)
    for sign in (-1, 1):
        ref = np.exp(sign * 2j * np.pi * np.outer(j, j) / N) @ f
        np.testing.assert_allclose(oracle.fft1d(f, sign), ref, rtol=0, atol=1e-12 * max(1, N))


@pytest.mark.parametrize("shape", [(2, 2, 2, 2), (3, 2, 3, 2), (6, 5, 4, 3)])
def test_fft4d_brute(shape):
    rng = np.random.default_rng(sum(shape))
    f = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    for sign in (-1, 1):
        np.testing.assert_allclose(oracle.fft4d(f, sign), brute_dft4(f, sign), rtol=0, atol=1e-11)


@pytest.mark.parametrize("shape", [(4, 4, 4, 4), (10, 8, 4, 6), (8, 8, 8, 8), (6, 9, 5, 7)])
def test_fft4d_numpy(shape):
    rng = np.random.default_rng(7)
    f = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    np.testing.assert_allclose(oracle.fft4d(f, -1), np.fft.fftn(f), rtol=0, atol=1e-10)
    np.testing.assert_allclose(oracle.fft4d(f, +1), np.fft.ifftn(f) * f.size, rtol=0, atol=1e-10)


def test_fft4d_closed_forms():
    shape = (4, 6, 2, 8)
    V = np.prod(shape)
    d = np.zeros(shape, dtype=np.complex128)
    d[0, 0, 0, 0] = 1
    np.testing.assert_allclose(oracle.fft4d(d, -1), np.ones(shape), atol=1e-14)
    # plane wave exp(+2 pi i k0.x/N) -> V at k0 under the forward (sign -1) transform
    k0 = (1, 5, 1, 3)
    grids = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    pw = np.exp(2j * np.pi * sum(k0[a] * grids[a] / shape[a] for a in range(4)))
    out = oracle.fft4d(pw, -1)
    ref = np.zeros(shape, dtype=np.complex128)
    ref[k0] = V
    np.testing.assert_allclose(out, ref, atol=1e-11)
    # Parseval
    rng = np.random.default_rng(3)
    f = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    F = oracle.fft4d(f, -1)
    assert abs(np.sum(abs(F) ** 2) / V - np.sum(abs(f) ** 2)) < 1e-12 * np.sum(abs(f) ** 2)
    # forward then backward is V times the identity
    np.testing.assert_allclose(oracle.fft4d(F, +1) / V, f, atol=1e-13)
