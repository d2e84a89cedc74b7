"""Pins for Delta (Eqs. 3, 5), theta (Eq. 4) and F (Eq. 1) in the oracle.

The decisive pin is the gradient identity derived from Eq. 1: for g(y) = exp(i omega^a T^a) at one
site y (T^a = lambda^a/2) and g = 1 elsewhere,
    dF/d omega^a |_0 = -(i / (24 V)) Tr[T^a Delta(y)],
checked by central finite differences of the oracle's own F. A wrong sign, a wrong neighbour
(x + nu instead of x - nu), a missing h.c. or trace term or a wrong factor fails it. Closed forms for
a one-link abelian configuration pin theta and F absolutely."""
import numpy as np
import pytest
import scipy.linalg

import oracle
import synth
from helpers import gell_mann, identity_links, random_su3


def test_delta_antihermitian_traceless_zero_sum():
    U = synth.config((4, 4, 6, 4), 3, 0.6)
    D = oracle.delta(U)
    np.testing.assert_allclose(D + np.conj(np.swapaxes(D, -1, -2)), 0, atol=1e-14)
    np.testing.assert_allclose(np.trace(D, axis1=-2, axis2=-1), 0, atol=1e-14)
    np.testing.assert_allclose(D.sum(axis=(0, 1, 2, 3)), 0, atol=1e-12)  # telescopes on a torus
    assert oracle.theta(D) > 0


def test_delta_vanishes_on_constant_links():
    dims = (4, 2, 3, 4)
    U = identity_links(dims)
    assert np.abs(oracle.delta(U)).max() == 0
    assert oracle.functional(U) == 1.0
    rng = np.random.default_rng(0)
    C = random_su3(rng, 4)
    for mu in range(4):
        U[mu] = C[mu]
    assert np.abs(oracle.delta(U)).max() < 1e-15


def test_one_link_closed_form():
    """All links 1 except U_x(x0) = diag(e^{i phi}, e^{-i phi}, 1):
    Delta(x0) = diag(-2i sin phi, 2i sin phi, 0) = -Delta(x0 + x-hat), zero elsewhere;
    theta = 16 sin^2(phi) / (3V);  F = 1 - (2 - 2 cos phi) / (12 V)."""
    dims = (4, 3, 2, 5)
    V = np.prod(dims)
    phi = 0.7
    U = identity_links(dims)
    x0 = (3, 1, 2, 2)  # (t, z, y, x)
    U[(0,) + x0] = np.diag([np.exp(1j * phi), np.exp(-1j * phi), 1])
    D = oracle.delta(U)
    expect = np.diag([-2j * np.sin(phi), 2j * np.sin(phi), 0])
    np.testing.assert_allclose(D[x0], expect, atol=1e-15)
    x1 = x0[:3] + ((x0[3] + 1) % dims[0],)
    np.testing.assert_allclose(D[x1], -expect, atol=1e-15)
    mask = np.ones(D.shape[:4], bool)
    mask[x0] = mask[x1] = False
    assert np.abs(D[mask]).max() == 0
    assert abs(oracle.theta(D) - 16 * np.sin(phi) ** 2 / (3 * V)) < 1e-16
    assert abs(oracle.functional(U) - (1 - (2 - 2 * np.cos(phi)) / (12 * V))) < 1e-15


@pytest.mark.parametrize("dims,seed", [((2, 3, 2, 3), 1), ((4, 4, 2, 2), 2)])
def test_gradient_identity_finite_differences(dims, seed):
    nx, ny, nz, nt = dims
    V = nx * ny * nz * nt
    U = synth.config(dims, seed, 0.5)
    D = oracle.delta(U)
    T = gell_mann() / 2
    rng = np.random.default_rng(seed)
    h = 1e-6
    for _ in range(4):
        y = tuple(int(rng.integers(0, n)) for n in (nt, nz, ny, nx))
        for a in range(8):
            def F_at(w):
                g = np.zeros(U.shape[1:], dtype=np.complex128)
                g[..., 0, 0] = g[..., 1, 1] = g[..., 2, 2] = 1
                g[y] = scipy.linalg.expm(1j * w * T[a])
                return oracle.functional(U, g)
            fd = (F_at(h) - F_at(-h)) / (2 * h)
            an = (-1j / (24 * V) * np.trace(T[a] @ D[y])).real
            assert abs(fd - an) < 1e-8 * max(1e-3, abs(an)) + 1e-10, (y, a, fd, an)


def test_functional_with_g_is_gauge_transform():
    """F_U[g] equals F evaluated on the transformed links (Eq. 1 read both ways)."""
    dims = (2, 4, 2, 2)
    U = synth.config(dims, 9, 0.4)
    rng = np.random.default_rng(5)
    g = random_su3(rng, int(np.prod(dims))).reshape(U.shape[1:])
    assert abs(oracle.functional(U, g) - oracle.functional(oracle.gauge_transform(U, g))) < 1e-14


def test_theta_scales_and_is_invariant_under_global_rotation():
    U = synth.config((4, 4, 4, 4), 4, 0.6)
    th = oracle.theta(oracle.delta(U))
    F = oracle.functional(U)
    U2 = synth.global_rotation(U.copy(), 77)
    assert abs(oracle.theta(oracle.delta(U2)) - th) < 1e-13 * th
    assert abs(oracle.functional(U2) - F) < 1e-13
