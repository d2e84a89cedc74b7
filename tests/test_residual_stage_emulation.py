"""The residual stage of the mixed schedule, emulated on the CPU at single precision with the oracle's steps:
past the handover, U = U_h + R with R a float residual starting at 0, Delta(U) = Delta(U_h) + Delta(R), the
update adds a U + (U + a U) b^+ to R with a = g(x) - 1, b = g(x + mu) - 1 formed by the small-step projection in
float and U read as float(U_h) + R, and H = 1 + K gathers the transformation. After a few iterations the tracked
links stay within 1e-10 of the oracle's double iterations from the same U_h, and the links rebuilt exactly as
proj(1 + K) U_h proj(1 + K)^+(x + mu) do too, so float arithmetic on the residual loses nothing that matters at
theta ~ 1e-15. CPU only."""
import numpy as np
import pytest

import oracle
import synth

HALF_ALPHA = 0.04


def shift_fwd(f, mu):
    """f(x + mu) for a site field of shape (Nt, Nz, Ny, Nx, ...), mu = 0..3 for x, y, z, t."""
    return np.roll(f, -1, axis=3 - mu)


def dagger(m):
    return np.conj(np.swapaxes(m, -1, -2))


def rsqrt1p_m1(t):
    return t * (-0.5 + t * (0.375 + t * -0.3125))


def small_step(X):
    """a = GS(1 + X) - 1 by the small-step formulas, site by site, in X's dtype (float here)."""
    a = np.zeros_like(X)
    x0, x1 = X[..., 0, :], X[..., 1, :]
    t0 = 2 * x0[..., 0].real + np.sum(np.abs(x0) ** 2, axis=-1)
    c0 = rsqrt1p_m1(t0)
    a[..., 0, :] = x0 * (1 + c0)[..., None]
    a[..., 0, 0] += c0
    a0 = a[..., 0, :]
    p = np.conj(a0[..., 1]) + x1[..., 0] + np.sum(np.conj(a0) * x1, axis=-1)
    d = x1 - p[..., None] * a0
    d[..., 0] -= p
    t1 = 2 * d[..., 1].real + np.sum(np.abs(d) ** 2, axis=-1)
    c1 = rsqrt1p_m1(t1)
    a[..., 1, :] = d * (1 + c1)[..., None]
    a[..., 1, 1] += c1
    r0, r1 = a[..., 0, :], a[..., 1, :]
    a[..., 2, 0] = np.conj(r0[..., 1] * r1[..., 2] - r0[..., 2] * r1[..., 1] - r0[..., 2])
    a[..., 2, 1] = np.conj(r0[..., 2] * r1[..., 0] - r0[..., 0] * r1[..., 2] - r1[..., 2])
    a[..., 2, 2] = np.conj(r0[..., 0] * r1[..., 1] - r0[..., 1] * r1[..., 0] + r1[..., 1] + r0[..., 0])
    return a


def test_shift_convention_matches_the_oracle_transform():
    U = synth.config((4, 4, 4, 6), 5, 0.6)
    g = oracle.gauge_field(oracle.fourier_filter(oracle.delta(U)), 0.08)
    mine = np.stack([g @ U[mu] @ dagger(shift_fwd(g, mu)) for mu in range(4)])
    assert np.abs(mine - oracle.gauge_transform(U, g)).max() < 1e-14


@pytest.mark.parametrize("theta_h,steps", [(1e-11, 6), (1e-7, 12)])
def test_float_residual_iterations_track_the_double_iterations(theta_h, steps):
    """From handover links at theta below theta_h; with theta_h = 1e-7 the links change by ~7e-5 over the
    stage, the size of the changes after the handover at 64^4."""
    dims = (4, 4, 4, 4)
    U0 = synth.config(dims, 3, 0.6)
    Uh = oracle.fix(U0, 0.08, theta_h, 500)[0]  # the handover links
    # the oracle's double iterations from U_h
    Uref = Uh.copy()
    for _ in range(steps):
        Uref = oracle.gauge_transform(Uref, oracle.gauge_field(oracle.fourier_filter(oracle.delta(Uref)), 0.08))
    # the residual stage at single precision
    Dh = oracle.delta(Uh)
    B = Uh.astype(np.complex64)
    R = np.zeros_like(B)
    K = np.zeros(Uh.shape[1:], dtype=np.complex64)
    for _ in range(steps):
        D = (Dh + oracle.delta(R.astype(np.complex128))).astype(np.complex64)
        X = (HALF_ALPHA * oracle.fourier_filter(D.astype(np.complex128))).astype(np.complex64)
        a = small_step(X)
        K = (a + K) + a @ K
        for mu in range(4):
            b = shift_fwd(a, mu)
            u = B[mu] + R[mu]
            t = a @ u
            R[mu] = R[mu] + (t + (u + t) @ dagger(b))
    assert R.dtype == np.complex64 and K.dtype == np.complex64
    tracked = Uh + R.astype(np.complex128)
    change = float(np.abs(Uref - Uh).max())
    assert change > 1e-7  # the stage moved the links
    assert np.abs(tracked - Uref).max() < 1e-10, (np.abs(tracked - Uref).max(), change)
    # the exact rebuild from the gathered transformation
    H = np.array([oracle.reunitarize(m) for m in (np.eye(3) + K.astype(np.complex128)).reshape(-1, 3, 3)])
    H = H.reshape(K.shape)
    rebuilt = oracle.gauge_transform(Uh, H)
    assert np.abs(rebuilt - Uref).max() < 1e-10
    th_ref, th_reb = oracle.theta(oracle.delta(Uref)), oracle.theta(oracle.delta(rebuilt))
    assert abs(th_reb - th_ref) < 1e-3 * th_ref, (th_reb, th_ref)
    assert abs(oracle.plaquette(rebuilt) - oracle.plaquette(U0)) < 1e-14
