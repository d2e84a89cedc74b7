"""FP64 CPU oracle for Fourier-accelerated Landau gauge fixing (Eqs. 1-5, Algorithm 1).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's CPU-baseline leg load
this module. The product path (the CUDA library and its binding) never imports it and shares no code
with it. oracle.c holds the arithmetic; this file is ctypes marshalling.

Array conventions: links complex128 (4, Nt, Nz, Ny, Nx, 3, 3); site matrix fields complex128
(Nt, Nz, Ny, Nx, 3, 3); scalar fields complex128 (Nt, Nz, Ny, Nx); dims = (Nx, Ny, Nz, Nt).
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force=False):
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp",
                               "-ffp-contract=off", src, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        P = ctypes.POINTER
        I4 = P(ctypes.c_int)
        vp, d, i, l = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_long
        lib.orc_delta.argtypes = [I4, vp, vp]
        lib.orc_theta.argtypes = [I4, vp]
        lib.orc_theta.restype = d
        lib.orc_functional.argtypes = [I4, vp, vp]
        lib.orc_functional.restype = d
        lib.orc_fft1d.argtypes = [i, vp, l, i]
        lib.orc_fft4d.argtypes = [I4, vp, i]
        lib.orc_p2.argtypes = [I4, I4]
        lib.orc_p2.restype = d
        lib.orc_p2max.argtypes = [I4]
        lib.orc_p2max.restype = d
        lib.orc_fourier_filter.argtypes = [I4, vp, vp]
        lib.orc_reunitarize.argtypes = [vp]
        lib.orc_gauge_field.argtypes = [I4, vp, d, vp]
        lib.orc_gauge_transform.argtypes = [I4, vp, vp]
        lib.orc_fix.argtypes = [I4, vp, d, d, i, vp, i, P(d), P(d)]
        lib.orc_fix.restype = i
        lib.orc_wilson_loop.argtypes = [I4, vp, i, i]
        lib.orc_wilson_loop.restype = d
        lib.orc_unitarity_violation.argtypes = [I4, vp, l]
        lib.orc_unitarity_violation.restype = d
        _lib = lib
    return _lib


def _c(a):
    assert a.dtype == np.complex128 and a.flags.c_contiguous, "complex128 C-contiguous arrays only"
    return a.ctypes.data


def dims_of_links(U):
    nt, nz, ny, nx = U.shape[1:5]
    return (nx, ny, nz, nt)


def dims_of_field(f):
    nt, nz, ny, nx = f.shape[0:4]
    return (nx, ny, nz, nt)


def _d(dims):
    return (ctypes.c_int * 4)(*[int(v) for v in dims])


def delta(U):
    """Eq. 5: Delta(x), shape (Nt, Nz, Ny, Nx, 3, 3)."""
    dims = dims_of_links(U)
    out = np.empty(U.shape[1:], dtype=np.complex128)
    _load().orc_delta(_d(dims), _c(U), _c(out))
    return out


def theta(Delta):
    """Eq. 4."""
    return _load().orc_theta(_d(dims_of_field(Delta)), _c(Delta))


def functional(U, g=None):
    """Eq. 1: F_U[g]; g=None means g = 1."""
    return _load().orc_functional(_d(dims_of_links(U)), _c(U), None if g is None else _c(g))


def fft1d(f, sign):
    f = np.ascontiguousarray(f, dtype=np.complex128).copy()
    _load().orc_fft1d(len(f), _c(f), 1, int(sign))
    return f


def fft4d(f, sign):
    """4D transform of a scalar field (Nt, Nz, Ny, Nx): sum_x f(x) exp(sign 2 pi i k.x/N)."""
    f = np.ascontiguousarray(f, dtype=np.complex128).copy()
    _load().orc_fft4d(_d(dims_of_field(f)), _c(f), int(sign))
    return f


def p2(dims, k):
    return _load().orc_p2(_d(dims), (ctypes.c_int * 4)(*[int(v) for v in k]))


def p2max(dims):
    return _load().orc_p2max(_d(dims))


def fourier_filter(Delta):
    """Algorithm 1, the FFT block: Delta-tilde = F^-1[(p2max/p2) F[Delta]] / V for every element."""
    out = np.empty_like(Delta)
    _load().orc_fourier_filter(_d(dims_of_field(Delta)), _c(Delta), _c(out))
    return out


def reunitarize(m):
    m = np.ascontiguousarray(m, dtype=np.complex128).reshape(3, 3).copy()
    _load().orc_reunitarize(_c(m))
    return m


def gauge_field(Dt, alpha):
    out = np.empty_like(Dt)
    _load().orc_gauge_field(_d(dims_of_field(Dt)), _c(Dt), float(alpha), _c(out))
    return out


def gauge_transform(U, g):
    """U_mu(x) -> g(x) U_mu(x) g^dagger(x+mu); returns a new array."""
    U = U.copy()
    _load().orc_gauge_transform(_d(dims_of_links(U)), _c(U), _c(g))
    return U


def fix(U, alpha=0.08, eps=1e-15, max_iter=100000, hist_len=0):
    """Algorithm 1. Returns (U_fixed, iters, theta, F, hist[(iters+1), 2])."""
    U = U.copy()
    th, F = ctypes.c_double(), ctypes.c_double()
    hist = np.zeros((max(hist_len, 1), 2), dtype=np.float64)
    it = _load().orc_fix(_d(dims_of_links(U)), _c(U), float(alpha), float(eps), int(max_iter),
                         hist.ctypes.data if hist_len > 0 else None, int(hist_len),
                         ctypes.byref(th), ctypes.byref(F))
    return U, it, th.value, F.value, hist[:min(it + 1, hist_len)] if hist_len > 0 else None


def wilson_loop(U, R, T):
    return _load().orc_wilson_loop(_d(dims_of_links(U)), _c(U), int(R), int(T))


def plaquette(U):
    return wilson_loop(U, 1, 1)


def unitarity_violation(U):
    return _load().orc_unitarity_violation(_d(dims_of_links(U)), _c(U), int(U.size // 9))
