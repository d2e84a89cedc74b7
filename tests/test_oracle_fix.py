"""Pins for the whole of Algorithm 1 in the oracle: F never decreases (beyond the roundoff of its own
sum), F <= 1, theta falls below eps, gauge-invariant loops and unitarity are kept, a pure-gauge field
reaches F = 1, and a global rotation of the input leaves the theta and F histories unchanged."""
import numpy as np

import oracle
import synth
from helpers import U_EPS


def _monotone(hist, V):
    floor = 64 * np.sqrt(4 * V) * U_EPS  # roundoff of the F sum over 4V links
    return np.all(np.diff(hist[:, 1]) >= -floor)


def test_fix_8_4_eps_03():
    dims = (8, 8, 8, 8)
    V = 8 ** 4
    U = synth.config(dims, 1, 0.3)
    Uf, it, th, F, hist = oracle.fix(U, 0.08, 1e-15, 1000, hist_len=1001)
    assert th < 1e-15 and 0 < it < 1000
    assert hist[-1, 0] == th and hist[-1, 1] == F
    assert np.all(hist[:-1, 0] >= 1e-15)  # the loop ran while theta >= eps
    assert _monotone(hist, V)
    assert F <= 1.0
    for R, T in [(1, 1), (1, 2), (2, 2)]:
        assert abs(oracle.wilson_loop(Uf, R, T) - oracle.wilson_loop(U, R, T)) < 1e-13
    assert oracle.unitarity_violation(Uf) < 1e-13
    # theta falls geometrically at the end (Fourier acceleration removes the slow modes)
    assert hist[-1, 0] < hist[-3, 0] * 0.5


def test_pure_gauge_near_identity_reaches_F1():
    dims = (4, 4, 4, 8)
    U = synth.config(dims, 3, 0.0, h_mode=synth.H_NEAR_IDENTITY, h_scale=0.5)
    assert abs(oracle.plaquette(U) - 1) < 1e-14
    Uf, it, th, F, hist = oracle.fix(U, 0.08, 1e-15, 2000, hist_len=2001)
    assert th < 1e-15
    assert abs(F - 1) < 1e-12
    assert _monotone(hist, np.prod(dims))


def test_pure_gauge_haar_converges():
    dims = (4, 4, 4, 4)
    U = synth.config(dims, 3, 0.0)
    Uf, it, th, F, hist = oracle.fix(U, 0.08, 1e-15, 5000, hist_len=5001)
    assert th < 1e-15 and F <= 1 + 1e-14
    assert _monotone(hist, np.prod(dims))


def test_diagonal_global_rotation_leaves_history_unchanged():
    """Gram-Schmidt projection commutes with conjugation by a diagonal SU(3) matrix, so a constant
    diagonal rotation of the input leaves the theta and F histories unchanged to roundoff."""
    dims = (4, 4, 6, 4)
    U = synth.config(dims, 12, 0.5)
    a, b = 0.37, -1.21
    d = np.array([np.exp(1j * a), np.exp(1j * b), np.exp(-1j * (a + b))])
    U2 = np.ascontiguousarray(d[:, None] * U * np.conj(d)[None, :])
    _, it1, _, _, h1 = oracle.fix(U, 0.08, 1e-15, 200, hist_len=201)
    _, it2, _, _, h2 = oracle.fix(U2, 0.08, 1e-15, 200, hist_len=201)
    n = min(len(h1), len(h2))
    assert abs(it1 - it2) <= 1
    np.testing.assert_allclose(h1[:n, 1], h2[:n, 1], rtol=0, atol=1e-13)
    big = h1[:n, 0] > 1e-6
    np.testing.assert_allclose(h1[:n][big, 0], h2[:n][big, 0], rtol=1e-10)


def test_general_global_rotation_agrees_to_second_order():
    """A general constant rotation commutes with the first-order step but not with the Gram-Schmidt
    projection, which differs at O(alpha^2 Delta^2): the F histories agree to that order and both
    runs converge."""
    dims = (4, 4, 6, 4)
    U = synth.config(dims, 12, 0.5)
    U2 = synth.global_rotation(U.copy(), 99)
    _, it1, th1, F1, h1 = oracle.fix(U, 0.08, 1e-15, 500, hist_len=501)
    _, it2, th2, F2, h2 = oracle.fix(U2, 0.08, 1e-15, 500, hist_len=501)
    assert th1 < 1e-15 and th2 < 1e-15
    np.testing.assert_allclose(h1[:3, 1], h2[:3, 1], rtol=0, atol=2e-3)
    assert abs(h1[1, 1] - h2[1, 1]) < 1e-3


def test_zero_iterations_when_converged():
    dims = (2, 2, 2, 2)
    U = synth.config(dims, 1, 0.0, h_mode=synth.H_IDENTITY)
    Uf, it, th, F, hist = oracle.fix(U, 0.08, 1e-15, 10, hist_len=11)
    assert it == 0 and th == 0.0 and F == 1.0
