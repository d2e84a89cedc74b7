"""Shared pieces of the GPU parity tests: tolerances and small helpers (no method arithmetic)."""
import numpy as np

U_EPS = 2.0 ** -53


def theta_tol(theta_ref):
    """|theta_gpu - theta_oracle| bound: 1e-12 relative plus an absolute roundoff floor 64 u sqrt(theta).
    Delta entries are differences of O(1) link entries with ~8u absolute error each, so theta's
    roundoff is about 2 sqrt(theta) 8u; relative 1e-12 alone is unreachable once theta < ~1e-6."""
    return 1e-12 * theta_ref + 64 * U_EPS * np.sqrt(theta_ref)


def assert_matrix_close(a, b, rtol=1e-12, scale=None):
    """Elementwise agreement relative to the matrix scale (SU(3) entries are O(1))."""
    if scale is None:
        scale = max(1.0, float(np.abs(b).max()))
    err = float(np.abs(a - b).max())
    assert err <= rtol * scale, "max abs err %.3e > %.1e * %.3e" % (err, rtol, scale)
    return err
