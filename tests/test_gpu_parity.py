"""Parity of the CUDA path (called through the C ABI) with the FP64 oracle, step by step and over
whole trajectories of Algorithm 1. Tolerances: 1e-12 relative to the O(1) matrix scale for links,
Delta, g; 1e-12 relative for F; theta within gpu_common.theta_tol."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import assert_matrix_close, theta_tol

pytestmark = pytest.mark.gpu

# generic FFT passes: 4^4, 6x4x8x10, 3x5x4x2, 12x6x5x9, 2^4; specialised passes: 8^4, 16x16x24x8,
# 24x24x8x48, 32x32x16x8
DIMS = [(4, 4, 4, 4), (8, 8, 8, 8), (6, 4, 8, 10), (3, 5, 4, 2), (12, 6, 5, 9), (2, 2, 2, 2), (16, 16, 24, 8),
        (24, 24, 8, 48), (32, 32, 16, 8)]


@pytest.fixture(scope="module")
def lgf():
    import torch
    assert torch.cuda.is_available()
    import paper_1210_8018_gb300 as m
    return m


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


@pytest.mark.parametrize("dims", DIMS)
def test_delta_theta_F(lgf, dims):
    U = synth.config(dims, 21, 0.6)
    D_ref = oracle.delta(U)
    th_ref, F_ref = oracle.theta(D_ref), oracle.functional(U)
    with lgf.Lattice(dims) as lat:
        out = np.empty_like(D_ref)
        th, F = lat.delta(U, out)  # host buffers
        assert_matrix_close(out, D_ref)
        assert abs(th - th_ref) <= theta_tol(th_ref)
        assert abs(F - F_ref) <= 1e-12 * abs(F_ref) + 1e-15
        # device buffers give the same bits
        outd = dev(np.zeros_like(D_ref))
        th2, F2 = lat.delta(dev(U), outd)
        assert np.array_equal(outd.cpu().numpy(), out) and th2 == th and F2 == F


@pytest.mark.parametrize("dims", DIMS)
def test_fourier_filter(lgf, dims):
    U = synth.config(dims, 22, 0.6)
    D = oracle.delta(U)
    Dt_ref = oracle.fourier_filter(D)
    with lgf.Lattice(dims) as lat:
        out = np.empty_like(D)
        lat.filter(D, out)
    assert_matrix_close(out, Dt_ref, scale=float(np.abs(Dt_ref).max()))


@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (16, 16, 24, 8), (24, 24, 8, 48)])
def test_fourier_filter_generic_passes(lgf, dims, monkeypatch):
    """The generic pass family on the shapes that normally take the specialised passes."""
    monkeypatch.setenv("LGF_GENERIC_FFT", "1")
    U = synth.config(dims, 25, 0.6)
    D = oracle.delta(U)
    Dt_ref = oracle.fourier_filter(D)
    with lgf.Lattice(dims) as lat:
        out = np.empty_like(D)
        lat.filter(D, out)
        out32 = np.empty_like(D)
        lat.filter(D, out32, "fp32")
    assert_matrix_close(out, Dt_ref, scale=float(np.abs(Dt_ref).max()))
    assert_matrix_close(out32, Dt_ref, rtol=5e-6, scale=float(np.abs(Dt_ref).max()))


@pytest.mark.parametrize("dims", [(8, 8, 8, 64), (16, 16, 32, 64)])
def test_float_t_filter_in_registers(lgf, dims, monkeypatch):
    """The float t pass with the filter held in registers (Nt = 64) applies the operations of the
    shared-memory tile pass in the same order: the filtered field is the same bits (LGF_TFILTER_REG=0 selects
    the tile pass), and it matches the oracle's filter to float accuracy."""
    U = synth.config(dims, 26, 0.6)
    D = oracle.delta(U)
    Dt_ref = oracle.fourier_filter(D)
    outs = []
    for flag in ("1", "0"):
        monkeypatch.setenv("LGF_TFILTER_REG", flag)
        with lgf.Lattice(dims) as lat:
            out = np.empty_like(D)
            lat.filter(D, out, "fp32")
        outs.append(out)
    assert np.array_equal(outs[0], outs[1])
    assert_matrix_close(outs[0], Dt_ref, rtol=5e-6, scale=float(np.abs(Dt_ref).max()))


@pytest.mark.parametrize("dims", [(6, 4, 8, 16), (16, 16, 16, 16)])
def test_float_delta_walking_t(lgf, dims, monkeypatch):
    """The float Delta that walks along t (the backward t link's combinations carried from the previous
    slice; forced on these small lattices with LGF_TWALK_MIN_BLOCKS=0) gives the same bits as the kernel in
    site order (LGF_TWALK=0); theta and F, summed over other groups of sites, agree to 1e-13."""
    monkeypatch.setenv("LGF_TWALK_MIN_BLOCKS", "0")
    U = synth.config(dims, 28, 0.6)
    res = []
    for flag in ("1", "0"):
        monkeypatch.setenv("LGF_TWALK", flag)
        with lgf.Lattice(dims) as lat:
            out = np.empty(U.shape[1:], dtype=np.complex128)
            th, F = lat.delta(U, out, "fp32")
        res.append((out, th, F))
    assert np.array_equal(res[0][0], res[1][0])
    assert abs(res[0][1] - res[1][1]) <= 1e-13 * res[1][1]
    assert abs(res[0][2] - res[1][2]) <= 1e-13


def test_float_xy_planes_in_registers(lgf, monkeypatch):
    """The float 64 x 64 xy passes held in registers apply the operations of the shared-memory tile passes
    in the same order: the filtered field is the same bits as with LGF_XY_REG=0, and matches the oracle."""
    dims = (64, 64, 8, 8)
    U = synth.config(dims, 27, 0.6)
    D = oracle.delta(U)
    Dt_ref = oracle.fourier_filter(D)
    outs = []
    for flag in ("1", "0"):
        monkeypatch.setenv("LGF_XY_REG", flag)
        with lgf.Lattice(dims) as lat:
            out = np.empty_like(D)
            lat.filter(D, out, "fp32")
        outs.append(out)
    assert np.array_equal(outs[0], outs[1])
    assert_matrix_close(outs[0], Dt_ref, rtol=5e-6, scale=float(np.abs(Dt_ref).max()))


@pytest.mark.parametrize("dims", DIMS)
def test_gauge_field(lgf, dims):
    U = synth.config(dims, 23, 0.6)
    Dt = oracle.fourier_filter(oracle.delta(U))
    g_ref = oracle.gauge_field(Dt, 0.08)
    with lgf.Lattice(dims) as lat:
        out = np.empty_like(Dt)
        lat.gauge(Dt, 0.08, out)
    assert_matrix_close(out, g_ref)


@pytest.mark.parametrize("dims", DIMS)
def test_gauge_update(lgf, dims):
    U = synth.config(dims, 24, 0.6)
    g = oracle.gauge_field(oracle.fourier_filter(oracle.delta(U)), 0.08)
    U_ref = oracle.gauge_transform(U, g)
    with lgf.Lattice(dims) as lat:
        Ud = dev(U)
        lat.update(Ud, dev(g))
        assert_matrix_close(Ud.cpu().numpy(), U_ref)


@pytest.mark.parametrize("dims,seed,eps", [((8, 8, 8, 8), 1, 0.3), ((6, 4, 8, 10), 5, 0.6), ((4, 4, 4, 8), 7, 0.6),
                                           ((16, 16, 8, 8), 8, 0.6)])
def test_trajectory_fp64(lgf, dims, seed, eps):
    """Whole fix: per-iteration theta and F histories, iteration count within +-1, final links."""
    U = synth.config(dims, seed, eps)
    Uo, it_o, th_o, F_o, h_o = oracle.fix(U, 0.08, 1e-15, 2000, hist_len=2001)
    Ud = dev(U)
    with lgf.Lattice(dims) as lat:
        r = lat.fix(Ud, 0.08, 1e-15, "fp64", history_len=2001)
    assert r["converged"] and r["theta"] < 1e-15
    assert abs(r["iters"] - it_o) <= 1
    h_g = r["history"]
    n = min(len(h_g), len(h_o))
    for k in range(n):
        assert abs(h_g[k, 1] - h_o[k, 1]) <= 1e-12 * abs(h_o[k, 1]), (k, h_g[k], h_o[k])
        assert abs(h_g[k, 0] - h_o[k, 0]) <= theta_tol(h_o[k, 0]), (k, h_g[k], h_o[k])
    assert_matrix_close(Ud.cpu().numpy(), Uo, rtol=1e-11)


@pytest.mark.parametrize("dims,seed,eps", [((8, 8, 8, 8), 1, 0.3), ((6, 4, 8, 10), 5, 0.6)])
def test_trajectory_plain_ieee_double_forms(lgf, dims, seed, eps, monkeypatch):
    """The double path with every step in plain IEEE double (the Fourier filter in double instead of
    double-float, no small-step forms): the same trajectory parity as the default forms, and the filter
    step itself."""
    monkeypatch.setenv("LGF_FFT_NATIVE_F64", "1")
    monkeypatch.setenv("LGF_SMALL_STEP", "0")
    U = synth.config(dims, seed, eps)
    D = oracle.delta(U)
    Dt_ref = oracle.fourier_filter(D)
    Uo, it_o, th_o, F_o, h_o = oracle.fix(U, 0.08, 1e-15, 2000, hist_len=2001)
    Ud = dev(U)
    with lgf.Lattice(dims) as lat:
        out = np.empty_like(D)
        lat.filter(D, out)
        r = lat.fix(Ud, 0.08, 1e-15, "fp64", history_len=2001)
    assert_matrix_close(out, Dt_ref, scale=float(np.abs(Dt_ref).max()))
    assert r["converged"] and r["theta"] < 1e-15
    assert abs(r["iters"] - it_o) <= 1
    h_g = r["history"]
    for k in range(min(len(h_g), len(h_o))):
        assert abs(h_g[k, 1] - h_o[k, 1]) <= 1e-12 * abs(h_o[k, 1]), (k, h_g[k], h_o[k])
        assert abs(h_g[k, 0] - h_o[k, 0]) <= theta_tol(h_o[k, 0]), (k, h_g[k], h_o[k])
    assert_matrix_close(Ud.cpu().numpy(), Uo, rtol=1e-11)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_host_links_give_the_device_result(lgf, precision):
    """Page-locked and pageable host links (staged through the context's buffers) give bitwise the result
    of the same fix on device links."""
    import torch
    dims = (8, 8, 8, 8)
    U = synth.config(dims, 2, 0.6)
    pinned = torch.from_numpy(U.copy()).pin_memory()
    pageable = U.copy()
    Ud = dev(U)
    with lgf.Lattice(dims) as lat:
        r_dev = lat.fix(Ud, 0.08, 1e-15, precision)
        r_pin = lat.fix(pinned.numpy(), 0.08, 1e-15, precision)
        r_pag = lat.fix(pageable, 0.08, 1e-15, precision)
    ref = Ud.cpu().numpy()
    assert r_dev["iters"] == r_pin["iters"] == r_pag["iters"]
    assert np.array_equal(pinned.numpy(), ref) and np.array_equal(pageable, ref)


def test_work_is_ordered_after_torchs_current_stream(lgf):
    """With torch tensors the library issues its work on torch's current stream, after what torch queued
    there: links produced on a side stream by a slow chain of kernels (zeros until the last one adds the
    configuration) are fixed as if they had been ready."""
    import torch
    dims = (32, 32, 16, 16)
    U = synth.config(dims, 3, 0.6)
    ref = dev(U)
    with lgf.Lattice(dims) as lat:
        r_ref = lat.fix(ref, 0.08, 1e-15, "mixed")
    src = dev(U)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        Us = torch.zeros_like(src)
        for _ in range(60):
            Us.mul_(1.0)
        Us.add_(src)
        with lgf.Lattice(dims) as lat:
            r = lat.fix(Us, 0.08, 1e-15, "mixed")
        out = Us.clone()
    torch.cuda.synchronize()
    assert r["iters"] == r_ref["iters"] and torch.equal(out, ref)


def test_one_step_parity_after_iterations(lgf):
    """Run k GPU iterations, hand the GPU's links to the oracle and compare one more iteration."""
    dims = (8, 6, 4, 10)
    U = synth.config(dims, 31, 0.6)
    with lgf.Lattice(dims) as lat:
        lat.load(dev(U), "fp64")
        lat.iterate(5, 0.08, 0.0)
        Uk = np.empty_like(U)
        lat.store(Uk)
        _, _, th_k, F_k, _ = oracle.fix(Uk, 0.08, 0.0, 0, hist_len=1)
        lat.load(Uk, "fp64")
        r = lat.iterate(1, 0.08, 0.0)
        U1 = np.empty_like(U)
        lat.store(U1)
    Uo, _, th_o, F_o, _ = oracle.fix(Uk, 0.08, 0.0, 1, hist_len=2)
    assert_matrix_close(U1, Uo)
    assert abs(r["F"] - F_o) <= 1e-12 * abs(F_o)
    assert abs(r["theta"] - th_o) <= theta_tol(th_o)


def test_gauge_invariants_and_unitarity(lgf):
    dims = (8, 8, 8, 8)
    U = synth.config(dims, 2, 0.6)
    Ud = dev(U)
    with lgf.Lattice(dims) as lat:
        m0 = lat.measure(Ud)
        lat.fix(Ud, 0.08, 1e-15, "fp64")
        m1 = lat.measure(Ud)
    Uf = Ud.cpu().numpy()
    assert abs(m0["plaquette"] - oracle.plaquette(U)) < 1e-14
    assert abs(m1["plaquette"] - m0["plaquette"]) < 1e-13
    for R, T in [(1, 2), (2, 2)]:
        assert abs(oracle.wilson_loop(Uf, R, T) - oracle.wilson_loop(U, R, T)) < 1e-13
    assert oracle.unitarity_violation(Uf) < 1e-13
    assert m1["theta"] < 1e-15


def test_pure_gauge_reaches_F1(lgf):
    dims = (8, 8, 8, 8)
    U = synth.config(dims, 3, 0.0, h_mode=synth.H_NEAR_IDENTITY, h_scale=0.5)
    with lgf.Lattice(dims) as lat:
        r = lat.fix(U, 0.08, 1e-15, "fp64")
    assert r["converged"] and abs(r["F"] - 1) < 1e-12


def test_already_converged_and_limits(lgf):
    dims = (4, 4, 4, 4)
    U = synth.config(dims, 1, 0.0, h_mode=synth.H_IDENTITY)
    with lgf.Lattice(dims) as lat:
        r = lat.fix(U, 0.08, 1e-15, "fp64")
        assert r["iters"] == 0 and r["theta"] == 0.0 and r["F"] == 1.0
        U2 = synth.config(dims, 4, 0.6)
        r = lat.fix(U2, 0.08, 1e-15, "fp64", max_iter=3)
        assert not r["converged"] and r["iters"] == 3


def test_error_paths(lgf):
    with pytest.raises(lgf.LgfError) as e:
        lgf.Lattice((7, 4, 4, 4))
    assert e.value.status == lgf.LGF_EINVAL
    with pytest.raises(lgf.LgfError):
        lgf.Lattice((1, 4, 4, 4))
    dims = (4, 4, 4, 4)
    U = synth.config(dims, 1, 0.5)
    U[0, 1, 2, 3, 0, 1, 1] = np.nan
    with lgf.Lattice(dims) as lat:
        with pytest.raises(lgf.LgfError) as e:
            lat.fix(U, 0.08, 1e-15)
        assert e.value.status == lgf.LGF_ENONFINITE
        # the context stays usable after a reported error
        r = lat.fix(synth.config(dims, 1, 0.5), 0.08, 1e-15)
        assert r["converged"]
