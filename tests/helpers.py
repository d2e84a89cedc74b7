"""Test-side utilities that are independent of both the oracle and the CUDA library.

They implement textbook operations (matrix exponentials through scipy, the lattice Laplacian through
numpy.roll, Gell-Mann generators), never the method's own steps.
"""
import numpy as np

U_EPS = np.finfo(np.float64).eps / 2  # unit roundoff u = 2^-53


def gell_mann():
    l = np.zeros((8, 3, 3), dtype=np.complex128)
    l[0][0, 1] = l[0][1, 0] = 1
    l[1][0, 1], l[1][1, 0] = -1j, 1j
    l[2][0, 0], l[2][1, 1] = 1, -1
    l[3][0, 2] = l[3][2, 0] = 1
    l[4][0, 2], l[4][2, 0] = -1j, 1j
    l[5][1, 2] = l[5][2, 1] = 1
    l[6][1, 2], l[6][2, 1] = -1j, 1j
    l[7] = np.diag([1, 1, -2]) / np.sqrt(3)
    return l


def laplacian(f):
    """(-d^2 f)(x) = sum_mu [2 f(x) - f(x+mu) - f(x-mu)] on a field indexed (t, z, y, x, ...)."""
    out = np.zeros_like(f)
    for ax in range(4):
        out += 2 * f - np.roll(f, -1, axis=ax) - np.roll(f, 1, axis=ax)
    return out


def random_su3(rng, n):
    """n Haar-ish SU(3) matrices via QR of complex Gaussians (test-side, numpy)."""
    z = rng.normal(size=(n, 3, 3)) + 1j * rng.normal(size=(n, 3, 3))
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=1, axis2=2)
    q = q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(q)
    q[:, :, 2] /= det[:, None]
    return q


def identity_links(dims):
    nx, ny, nz, nt = dims
    U = np.zeros((4, nt, nz, ny, nx, 3, 3), dtype=np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1
    return U


def site_index(dims, x, y, z, t):
    nx, ny, nz, nt = dims
    return (t, z, y, x)
