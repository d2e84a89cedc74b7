"""Arithmetic forms of the FP64 path that differ from a plain FP64 evaluation.

Delta (Eq. 5) is summed in 64-bit fixed point: checked against an extended-precision (long double)
evaluation of the same sum, where it must be at least as accurate as the oracle's FP64 sum.

The gauge update U_mu(x) -> g(x) U_mu(x) g^+(x+mu) (Algorithm 1) has two forms. Small step: with
a = g(x) - 1 and b = g(x+mu) - 1, the kernel adds delta = a U + (U + a U) b^+, formed in double-float
arithmetic, to rows 0 and 1 of U in FP64; a warp takes it when every element of a and b is below 2^-7.
General step: rows 0 and 1 by FP64 products. Both rebuild row 2 as conj(row0 x row1) in FP64, where the
oracle multiplies it out. Both are compared with the oracle's gauge transformation at the level of FP64
rounding (2e-15 absolute on O(1) entries for rows 0 and 1 of the small step, 1e-14 for whole links), far
tighter than the 1e-12 of the other parity tests; the environment switch LGF_SMALL_STEP=0 shows that the
default really runs the other arithmetic (the results differ in the last bits).

The projection g = SU(3)-projection of 1 + X, X = (alpha/2) Delta-tilde (Eq. 3), has a small-step form too
(g = 1 + a with a formed in double-float from small quantities) when every |X_ij| < 2^-8."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lgf():
    import torch
    assert torch.cuda.is_available()
    import paper_1210_8018_gb300 as m
    return m


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def near_identity_gauge(U, size):
    """g = GS(1 + X) with X = s Delta(U) anti-Hermitian traceless and max |X_ij| = size."""
    D = oracle.delta(U)
    return oracle.gauge_field(D, 2.0 * size / float(np.abs(D).max()))


def small_step(monkeypatch, on):
    if on:
        monkeypatch.delenv("LGF_SMALL_STEP", raising=False)
    else:
        monkeypatch.setenv("LGF_SMALL_STEP", "0")


def run_update(lgf, dims, U, g, monkeypatch, product_only):
    small_step(monkeypatch, not product_only)
    with lgf.Lattice(dims) as lat:
        Ud = dev(U)
        lat.update(Ud, dev(g))
        return Ud.cpu().numpy()


@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (3, 5, 4, 2), (16, 8, 6, 10)])
@pytest.mark.parametrize("size", [1e-6, 1e-3, 7e-3])
def test_small_step_form_at_fp64_rounding(lgf, dims, size, monkeypatch):
    U = synth.config(dims, 41, 0.6)
    g = near_identity_gauge(U, size)
    assert float(np.abs(g - np.eye(3)).max()) < 2.0 ** -7
    U_ref = oracle.gauge_transform(U, g)
    small = run_update(lgf, dims, U, g, monkeypatch, False)
    prod = run_update(lgf, dims, U, g, monkeypatch, True)
    e_rows01 = float(np.abs(small[..., :2, :] - U_ref[..., :2, :]).max())
    e_small = float(np.abs(small - U_ref).max())
    e_prod = float(np.abs(prod - U_ref).max())
    assert e_rows01 <= 2e-15, e_rows01  # the double-float correction itself
    assert e_small <= 1e-14, e_small    # row 2 = conj(row0 x row1), as in the product form
    assert e_prod <= 1e-14, e_prod
    assert not np.array_equal(small, prod)  # the default took the double-float form
    # the step itself (U' - U) is reproduced to a relative precision far beyond float
    step = U_ref - U
    assert float(np.abs((small - U)[..., :2, :] - step[..., :2, :]).max()) <= 2e-15
    # unitarity is kept at FP64 level
    uu = np.einsum("...ij,...kj->...ik", small, small.conj()) - np.eye(3)
    assert float(np.abs(uu).max()) < 1e-14


@pytest.mark.parametrize("split", ["00", "21", "44", "13"])
def test_general_form_fixed_point_and_fp64_splits(lgf, split, monkeypatch):
    """Large steps (Haar-random g): the general form splits a site's four directions between FP64 products and
    61-bit fixed-point products (LGF_UPDATE_SPLIT: FP64 directions in even and odd warps). Every split agrees
    with the oracle's gauge transformation at the FP64 rounding level of the product form."""
    monkeypatch.setenv("LGF_UPDATE_SPLIT", split)
    dims = (8, 8, 8, 8)
    U = synth.config(dims, 45, 0.6)
    g = np.ascontiguousarray(synth.config(dims, 46, 0.0)[0])  # random SU(3) matrices h(x) h^+(x + x-hat)
    U_ref = oracle.gauge_transform(U, g)
    out = run_update(lgf, dims, U, g, monkeypatch, False)  # no warp is small: every link takes the general form
    assert float(np.abs(out - U_ref).max()) <= 1e-14
    uu = np.einsum("...ij,...kj->...ik", out, out.conj()) - np.eye(3)
    assert float(np.abs(uu).max()) < 1e-14


@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (3, 5, 4, 2)])
def test_mixed_warps(lgf, dims, monkeypatch):
    """Small g everywhere except Haar-random g on the x = 0 sites of every other (y, z, t) row: warps
    containing such a site take the general form, the others the small-step form."""
    U = synth.config(dims, 43, 0.6)
    g = near_identity_gauge(U, 3e-3)
    H = synth.config(dims, 44, 0.0)[0]  # Haar h(x) h^+(x + x-hat) products: random SU(3) matrices
    nt, nz, ny, nx = U.shape[1:5]
    rows = np.arange(nt * nz * ny).reshape(nt, nz, ny) % 2 == 0
    g[..., 0, :, :][rows] = H[..., 0, :, :][rows]
    U_ref = oracle.gauge_transform(U, g)
    out = run_update(lgf, dims, U, g, monkeypatch, False)
    assert float(np.abs(out - U_ref).max()) <= 1e-14


@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (3, 5, 4, 2)])
@pytest.mark.parametrize("size", [1e-7, 1e-4, 3e-3])
def test_small_step_projection(lgf, dims, size, monkeypatch):
    U = synth.config(dims, 47, 0.6)
    Dt = oracle.fourier_filter(oracle.delta(U))
    alpha = 2.0 * size / float(np.abs(Dt).max())  # max |X_ij| = size
    g_ref = oracle.gauge_field(Dt, alpha)
    out = {}
    for on in (True, False):
        small_step(monkeypatch, on)
        with lgf.Lattice(dims) as lat:
            g = np.empty_like(Dt)
            lat.gauge(Dt, alpha, g)
            out[on] = g
    e_small = float(np.abs(out[True] - g_ref).max())
    e_gs = float(np.abs(out[False] - g_ref).max())
    assert e_small <= 1e-15, e_small
    assert e_gs <= 1e-15, e_gs
    assert not np.array_equal(out[True], out[False])
    uu = np.einsum("...ij,...kj->...ik", out[True], out[True].conj()) - np.eye(3)
    assert float(np.abs(uu).max()) < 2e-15
    det = np.linalg.det(out[True])
    assert float(np.abs(det - 1).max()) < 2e-15


def delta_extended(U):
    """Eq. 5 in long double: B = sum_nu [U_nu(x - nu) - U_nu(x)], Delta = B - B^+ - (1/3) Tr(B - B^+)."""
    re = U.real.astype(np.longdouble)
    im = U.imag.astype(np.longdouble)
    Br = np.zeros(U.shape[1:], dtype=np.longdouble)
    Bi = np.zeros(U.shape[1:], dtype=np.longdouble)
    for mu in range(4):
        ax = 3 - mu  # U[mu] has axes (t, z, y, x, 3, 3); direction mu = 0 is x
        Br += np.roll(re[mu], 1, axis=ax) - re[mu]
        Bi += np.roll(im[mu], 1, axis=ax) - im[mu]
    Dr = Br - np.swapaxes(Br, -1, -2)
    Di = Bi + np.swapaxes(Bi, -1, -2)
    tr = (Di[..., 0, 0] + Di[..., 1, 1] + Di[..., 2, 2]) / 3
    for k in range(3):
        Di[..., k, k] -= tr
    return Dr, Di


@pytest.mark.parametrize("dims,seed,eps", [((8, 8, 8, 8), 1, 0.3), ((6, 4, 8, 10), 45, 0.6), ((3, 5, 4, 2), 46, 0.6)])
def test_delta_fixed_point_accuracy(lgf, dims, seed, eps):
    U = synth.config(dims, seed, eps)
    Dr, Di = delta_extended(U)
    with lgf.Lattice(dims) as lat:
        out = np.empty(U.shape[1:], dtype=np.complex128)
        lat.delta(U, out)
    Do = oracle.delta(U)
    err_gpu = np.maximum(np.abs(out.real - Dr), np.abs(out.imag - Di)).astype(np.float64)
    err_orc = np.maximum(np.abs(Do.real - Dr), np.abs(Do.imag - Di)).astype(np.float64)
    mag = np.maximum(np.abs(Dr), np.abs(Di)).astype(np.float64).max(axis=(-1, -2), keepdims=True)
    # 16 link entries per element, each quantised to 2^-56 at most; then the roundings of the conversion to
    # double and of the diagonal (Delta_22 = -(Delta_00 + Delta_11)), relative to the site's largest entry
    assert float((err_gpu - 6 * 2.0 ** -53 * mag).max()) <= 16 * 2.0 ** -56
    assert float(np.sqrt((err_gpu ** 2).mean())) <= float(np.sqrt((err_orc ** 2).mean()))
