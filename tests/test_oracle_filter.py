"""Pins for p^2, p^2_max and the Fourier filter of Algorithm 1 (Eq. 2): the symbol of the lattice
Laplacian (numpy.roll, independent of the oracle), the maximum by enumeration, and the identity
-d^2 (filtered f) = p^2_max (f - mean f) that holds for any field."""
import itertools

import numpy as np
import pytest

import oracle
from helpers import laplacian


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 8, 10), (3, 5, 4, 7)])
def test_p2_is_laplacian_eigenvalue(dims):
    nx, ny, nz, nt = dims
    rng = np.random.default_rng(1)
    grids = np.meshgrid(np.arange(nt), np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for _ in range(6):
        k = [int(rng.integers(0, n)) for n in dims]  # (kx, ky, kz, kt)
        ph = (k[0] * grids[3] / nx + k[1] * grids[2] / ny + k[2] * grids[1] / nz + k[3] * grids[0] / nt)
        pw = np.exp(2j * np.pi * ph)
        lap = laplacian(pw)
        np.testing.assert_allclose(lap, oracle.p2(dims, k) * pw, atol=1e-12)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (3, 5, 4, 7), (8, 6, 2, 5)])
def test_p2max_is_max(dims):
    best = max(oracle.p2(dims, k) for k in itertools.product(*[range(n) for n in dims]))
    assert abs(oracle.p2max(dims) - best) < 1e-14
    if all(n % 2 == 0 for n in dims):
        assert abs(oracle.p2max(dims) - 16.0) < 1e-13


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 8, 10), (3, 5, 4, 7)])
def test_filter_inverts_laplacian(dims):
    """Filtered field h = F^-1 (p2max/p2) F f / V satisfies -d^2 h = p2max (f - <f>) elementwise."""
    nx, ny, nz, nt = dims
    rng = np.random.default_rng(11)
    f = rng.normal(size=(nt, nz, ny, nx, 3, 3)) + 1j * rng.normal(size=(nt, nz, ny, nx, 3, 3))
    h = oracle.fourier_filter(f)
    lhs = laplacian(h)
    rhs = oracle.p2max(dims) * (f - f.mean(axis=(0, 1, 2, 3), keepdims=True))
    np.testing.assert_allclose(lhs, rhs, atol=1e-11)
    # the zero mode is removed
    np.testing.assert_allclose(h.mean(axis=(0, 1, 2, 3)), 0, atol=1e-13)


def test_filter_keeps_antihermitian_traceless():
    import synth
    U = synth.config((4, 6, 4, 2), 5, 0.5)
    D = oracle.delta(U)
    Dt = oracle.fourier_filter(D)
    np.testing.assert_allclose(Dt + np.conj(np.swapaxes(Dt, -1, -2)), 0, atol=1e-13)
    np.testing.assert_allclose(np.trace(Dt, axis1=-2, axis2=-1), 0, atol=1e-13)


def test_filter_constant_mode_field():
    """A single Fourier mode passes through multiplied by exactly p2max/p2(k)."""
    dims = (4, 6, 4, 8)
    nx, ny, nz, nt = dims
    k = (1, 2, 3, 5)
    grids = np.meshgrid(np.arange(nt), np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    pw = np.exp(2j * np.pi * (k[0] * grids[3] / nx + k[1] * grids[2] / ny + k[2] * grids[1] / nz
                              + k[3] * grids[0] / nt))
    f = np.zeros((nt, nz, ny, nx, 3, 3), dtype=np.complex128)
    f[..., 1, 2] = pw
    h = oracle.fourier_filter(f)
    np.testing.assert_allclose(h[..., 1, 2], oracle.p2max(dims) / oracle.p2(dims, k) * pw, atol=1e-12)
    np.testing.assert_allclose(h[..., 0, 0], 0, atol=1e-14)
