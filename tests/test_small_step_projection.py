"""The small-step form of the SU(3) projection g = GS(1 + X) (X anti-Hermitian and traceless, small), written as
g = 1 + a with a formed from small quantities only: the double path forms a in double-float, the residual stage
of the mixed schedule in float. The formulas, emulated here in numpy at double and at single precision, are
checked against a textbook Gram-Schmidt of 1 + X in 40-digit arithmetic (and against the oracle's projection):
a matches GS(1 + X) - 1 to the working precision relative to |a|, for every |X_ij| up to 2^-8, so the
truncated series for (1 + t)^(-1/2) - 1 costs nothing at either precision. CPU only."""
import numpy as np
import pytest

import oracle

mpmath = pytest.importorskip("mpmath")


def rsqrt1p_m1(t):
    return t * (-0.5 + t * (0.375 + t * -0.3125))


def small_step(X):
    """a = GS(1 + X) - 1 by the small-step formulas, in X's dtype (rows 0-1, row 2 from them)."""
    dt = X.dtype
    a = np.zeros((3, 3), dtype=dt)
    x0, x1 = X[0], X[1]
    t0 = 2 * x0[0].real + np.sum(np.abs(x0) ** 2)
    c0 = rsqrt1p_m1(t0)
    s0 = 1 + c0
    a[0] = x0 * s0
    a[0, 0] += c0
    p = np.conj(a[0, 1]) + x1[0] + np.sum(np.conj(a[0]) * x1)
    d = x1 - p * a[0]
    d[0] -= p
    t1 = 2 * d[1].real + np.sum(np.abs(d) ** 2)
    c1 = rsqrt1p_m1(t1)
    s1 = 1 + c1
    a[1] = d * s1
    a[1, 1] += c1
    a[2, 0] = np.conj(a[0, 1] * a[1, 2] - a[0, 2] * a[1, 1] - a[0, 2])
    a[2, 1] = np.conj(a[0, 2] * a[1, 0] - a[0, 0] * a[1, 2] - a[1, 2])
    a[2, 2] = np.conj(a[0, 0] * a[1, 1] - a[0, 1] * a[1, 0] + a[1, 1] + a[0, 0])
    return a.astype(dt)


def exact_a(x):
    """GS(1 + X) - 1 in 40-digit arithmetic: rows 0-1 orthonormalised, row 2 = conj(row0 x row1)."""
    mp = mpmath.mp
    mp.dps = 40
    m = [[mpmath.mpc(complex(x[i, j])) + (1 if i == j else 0) for j in range(3)] for i in range(3)]
    n0 = mpmath.sqrt(sum(abs(v) ** 2 for v in m[0]))
    r0 = [v / n0 for v in m[0]]
    p = sum(mpmath.conj(a) * b for a, b in zip(r0, m[1]))
    r1 = [b - p * a for a, b in zip(r0, m[1])]
    n1 = mpmath.sqrt(sum(abs(v) ** 2 for v in r1))
    r1 = [v / n1 for v in r1]
    r2 = [mpmath.conj(r0[1] * r1[2] - r0[2] * r1[1]), mpmath.conj(r0[2] * r1[0] - r0[0] * r1[2]),
          mpmath.conj(r0[0] * r1[1] - r0[1] * r1[0])]
    rows = [r0, r1, r2]
    return [[rows[i][j] - (1 if i == j else 0) for j in range(3)] for i in range(3)]


def rel_err(a, ex):
    amax = max(abs(v) for row in ex for v in row)
    return float(max(abs(mpmath.mpc(complex(a[i, j])) - ex[i][j]) for i in range(3) for j in range(3)) / amax)


def random_x(rng, scale):
    h = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
    h = h + h.conj().T
    h -= np.trace(h) / 3 * np.eye(3)
    x = 1j * h
    return x * (scale / np.abs(x).max())


def test_small_step_matches_gram_schmidt():
    rng = np.random.default_rng(11)
    worst64 = worst32 = 0.0
    for scale in [2.0 ** -8, 2.0 ** -9, 2.0 ** -12, 1e-5, 1e-8]:
        for _ in range(60):
            x = random_x(rng, scale * rng.uniform(0.5, 1.0))
            ex = exact_a(x)
            worst64 = max(worst64, rel_err(small_step(x.astype(np.complex128)), ex))
            worst32 = max(worst32, rel_err(small_step(x.astype(np.complex64)), ex))
    assert worst64 < 2e-15, worst64
    assert worst32 < 2e-6, worst32


def test_small_step_agrees_with_the_oracle_projection():
    rng = np.random.default_rng(12)
    for _ in range(100):
        x = random_x(rng, 2.0 ** -9)
        g = oracle.reunitarize((np.eye(3) + x).reshape(1, 3, 3)).reshape(3, 3)
        assert np.abs((np.eye(3) + small_step(x)) - g).max() < 1e-15
