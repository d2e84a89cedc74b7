"""Pins for g(x) (first-order expansion plus SU(3) projection, Eq. 2 and the text after Eq. 3) and
the gauge update U -> g U g^dagger(x+mu) of Algorithm 1: unitarity, det = 1, idempotence, agreement
with scipy's matrix exponential to first order, and gauge invariance of Wilson loops whose values
are pinned by closed forms."""
import numpy as np
import pytest
import scipy.linalg

import oracle
import synth
from helpers import gell_mann, identity_links, random_su3


def test_reunitarize_gives_su3_and_is_idempotent():
    rng = np.random.default_rng(1)
    for m in rng.normal(size=(20, 3, 3)) + 1j * rng.normal(size=(20, 3, 3)):
        r = oracle.reunitarize(m)
        np.testing.assert_allclose(r @ r.conj().T, np.eye(3), atol=1e-15)
        assert abs(np.linalg.det(r) - 1) < 1e-15
        np.testing.assert_allclose(oracle.reunitarize(r), r, atol=1e-15)
    for h in random_su3(rng, 10):
        np.testing.assert_allclose(oracle.reunitarize(h), h, atol=2e-15)


def test_reunitarize_closed_form_diagonal():
    phi = 0.3
    r = oracle.reunitarize(np.diag([1 + 1j * phi, 1 - 1j * phi, 1]))
    z = (1 + 1j * phi) / abs(1 + 1j * phi)
    np.testing.assert_allclose(r, np.diag([z, np.conj(z), 1]), atol=1e-16)


def test_first_order_projection_matches_exponential():
    """GS(1 + X) = exp(X) + O(X^2) for anti-Hermitian traceless X."""
    rng = np.random.default_rng(2)
    T = gell_mann() / 2
    for scale in (1e-2, 1e-3, 1e-4):
        X = 1j * np.einsum("a,aij->ij", rng.normal(size=8), T) * scale
        err = np.abs(oracle.reunitarize(np.eye(3) + X) - scipy.linalg.expm(X)).max()
        assert err < 3 * scale ** 2, (scale, err)


def test_gauge_field_su3():
    U = synth.config((4, 2, 4, 2), 6, 0.6)
    g = oracle.gauge_field(oracle.fourier_filter(oracle.delta(U)), 0.08)
    gg = np.einsum("...ij,...kj->...ik", g, g.conj())
    np.testing.assert_allclose(gg, np.broadcast_to(np.eye(3), gg.shape), atol=1e-15)
    np.testing.assert_allclose(np.linalg.det(g), 1, atol=1e-15)


def abelian_field(dims, m):
    """U_y(x) = diag(e^{i f x}, e^{-i f x}, 1) with f = 2 pi m / Nx (all other links 1): a constant
    field strength f in the x-y plane, so an R x T loop in that plane equals (2 cos(R T f) + 1)/3."""
    nx = dims[0]
    f = 2 * np.pi * m / nx
    U = identity_links(dims)
    for x in range(nx):
        U[1, :, :, :, x] = np.diag([np.exp(1j * f * x), np.exp(-1j * f * x), 1])
    return U, f


@pytest.mark.parametrize("R,T", [(1, 1), (1, 2), (2, 1), (2, 2)])
def test_wilson_loop_closed_form(R, T):
    dims = (6, 4, 4, 4)
    U, f = abelian_field(dims, 1)
    # planes (x,y) and (y,x) carry the flux; the other ten ordered planes are trivial
    expect = (10 + 2 * (2 * np.cos(R * T * f) + 1) / 3) / 12
    if (R, T) in [(1, 2), (2, 1)]:
        expect = (10 + 2 * (2 * np.cos(2 * f) + 1) / 3) / 12
    assert abs(oracle.wilson_loop(U, R, T) - expect) < 1e-14


def test_gauge_transform_keeps_loops_and_unitarity():
    dims = (4, 4, 2, 4)
    U = synth.config(dims, 8, 0.6)
    rng = np.random.default_rng(3)
    g = random_su3(rng, int(np.prod(dims))).reshape(U.shape[1:])
    U2 = oracle.gauge_transform(U, g)
    for R, T in [(1, 1), (1, 2), (2, 2)]:
        assert abs(oracle.wilson_loop(U2, R, T) - oracle.wilson_loop(U, R, T)) < 1e-14
    assert oracle.unitarity_violation(U2) < 1e-14
    # undoing the transformation restores U
    gd = np.conj(np.swapaxes(g, -1, -2)).copy()
    np.testing.assert_allclose(oracle.gauge_transform(U2, gd), U, atol=1e-14)


def test_pure_gauge_field_from_identity():
    dims = (2, 2, 4, 2)
    rng = np.random.default_rng(4)
    h = random_su3(rng, int(np.prod(dims))).reshape((2, 4, 2, 2, 3, 3))
    U = oracle.gauge_transform(identity_links(dims), h)
    assert abs(oracle.plaquette(U) - 1) < 1e-14
    assert abs(oracle.functional(U, np.conj(np.swapaxes(h, -1, -2)).copy()) - 1) < 1e-14


def test_gauge_field_closed_form_half_alpha():
    """Delta-tilde = diag(i phi, -i phi, 0) gives g = diag(z, conj z, 1), z = (1 + i alpha phi/2)/|.|:
    pins the alpha/2 of the first-order expansion."""
    dims = (2, 2, 2, 2)
    phi, alpha = 0.9, 0.08
    Dt = np.zeros((2, 2, 2, 2, 3, 3), dtype=np.complex128)
    Dt[..., 0, 0], Dt[..., 1, 1] = 1j * phi, -1j * phi
    g = oracle.gauge_field(Dt, alpha)
    z = (1 + 0.5j * alpha * phi) / abs(1 + 0.5j * alpha * phi)
    np.testing.assert_allclose(g, np.broadcast_to(np.diag([z, np.conj(z), 1]), g.shape), atol=1e-16)


def test_unitarity_violation_detects():
    U = synth.config((2, 2, 2, 2), 1, 0.5)
    assert oracle.unitarity_violation(U) < 1e-14
    U[2, 1, 0, 1, 0] *= 1.001
    assert 1e-3 < oracle.unitarity_violation(U) < 1e-2
