"""Seeded synthetic SU(3) gauge configurations (inputs for tests and benchmarks).

U_mu(x) = h(x) exp(i eps A_mu(x)) h^dagger(x + mu), with A_mu^a ~ N(0,1) over the eight Gell-Mann
generators (normalised lambda^a / (2 sqrt 2)) and h(x) Haar-random on SU(3). eps = 0 is a pure-gauge
field. Random numbers come from Philox4x32-10, one counter per site and link, so the bytes do not depend
on the thread count. This module draws inputs only; it contains none of the gauge-fixing arithmetic.

Arrays use the links layout of the library: complex128, shape (4, Nt, Nz, Ny, Nx, 3, 3), C order.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libsynth.so")
_lib = None

H_HAAR, H_NEAR_IDENTITY, H_IDENTITY = 0, 1, 2
ALGEBRA_NORM = 1.0 / (2.0 * np.sqrt(2.0))


def build(force=False):
    """Compile synth.c into libsynth.so (plain C, OpenMP)."""
    src = os.path.join(_HERE, "synth.c")
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
        lib.synth_config.argtypes = [P(ctypes.c_int), ctypes.c_uint64, ctypes.c_double, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_void_p]
        lib.synth_global_rotation.argtypes = [P(ctypes.c_int), ctypes.c_uint64, ctypes.c_void_p]
        lib.synth_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_long, ctypes.c_double,
                                      ctypes.c_void_p]
        lib.synth_philox4x32_10.argtypes = [P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint32)]
        _lib = lib
    return _lib


def _dims_arg(dims):
    nx, ny, nz, nt = (int(d) for d in dims)
    return (ctypes.c_int * 4)(nx, ny, nz, nt)


def links_shape(dims):
    nx, ny, nz, nt = dims
    return (4, nt, nz, ny, nx, 3, 3)


def config(dims, seed, eps, h_mode=H_HAAR, h_scale=0.5, algebra_norm=ALGEBRA_NORM, out=None):
    """Return U (complex128, (4, Nt, Nz, Ny, Nx, 3, 3)); dims = (Nx, Ny, Nz, Nt).

    `out` may be a preallocated C-contiguous complex128 array of that shape (e.g. pinned memory)."""
    lib = _load()
    if out is None:
        out = np.empty(links_shape(dims), dtype=np.complex128)
    assert out.dtype == np.complex128 and out.flags.c_contiguous and out.shape == links_shape(dims)
    lib.synth_config(_dims_arg(dims), ctypes.c_uint64(seed), float(eps), int(h_mode), float(h_scale),
                     float(algebra_norm), out.ctypes.data)
    return out


def global_rotation(U, seed):
    """Apply one Haar-random constant gauge rotation to every link of U, in place."""
    lib = _load()
    nt, nz, ny, nx = U.shape[1:5]
    lib.synth_global_rotation(_dims_arg((nx, ny, nz, nt)), ctypes.c_uint64(seed), U.ctypes.data)
    return U


def normals(seed, stream, count, scale=1.0):
    lib = _load()
    out = np.empty(int(count), dtype=np.float64)
    lib.synth_normals(ctypes.c_uint64(seed), ctypes.c_uint32(stream), int(count), float(scale), out.ctypes.data)
    return out


def philox4x32_10(ctr, key):
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    lib.synth_philox4x32_10(c, k, o)
    return list(o)
