"""The float and mixed-precision schedules against the FP64 oracle: float single steps to float
accuracy, and a mixed fix that reaches theta < 1e-15 in double precision with links that stay exactly
gauge-equivalent to the input (plaquette and Wilson loops to 1e-14)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import assert_matrix_close

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


@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (6, 4, 8, 10)])
def test_fp32_steps(lgf, dims):
    """Float steps: error bounded by float roundoff (u32 = 6e-8) times small constants."""
    U = synth.config(dims, 41, 0.6)
    D = oracle.delta(U)
    Dt = oracle.fourier_filter(D)
    g = oracle.gauge_field(Dt, 0.08)
    with lgf.Lattice(dims) as lat:
        out = np.empty_like(D)
        th, F = lat.delta(U, out, "fp32")
        assert_matrix_close(out, D, rtol=2e-6)
        assert abs(F - oracle.functional(U)) < 1e-6
        lat.filter(D, out, "fp32")
        assert_matrix_close(out, Dt, rtol=5e-6, scale=float(np.abs(Dt).max()))
        lat.gauge(Dt, 0.08, out, "fp32")
        assert_matrix_close(out, g, rtol=1e-6)
        U2 = U.copy()
        lat.update(U2, g, "fp32")
        assert_matrix_close(U2, oracle.gauge_transform(U, g), rtol=2e-6)


@pytest.mark.parametrize("dims,seed,eps", [((8, 8, 8, 8), 1, 0.3), ((16, 16, 16, 16), 7, 0.6)])
def test_mixed_fix(lgf, dims, seed, eps):
    U = synth.config(dims, seed, eps)
    Ud = dev(U)
    with lgf.Lattice(dims) as lat:
        r = lat.fix(Ud, 0.08, 1e-15, "mixed", history_len=4000)
        m = lat.measure(Ud)
    Uf = Ud.cpu().numpy()
    assert r["converged"] and r["theta"] < 1e-15
    assert m["theta"] < 1e-15 and abs(m["F"] - r["F"]) < 1e-14
    # exact gauge equivalence with the input (double handover from the saved input)
    for R, T in [(1, 1), (1, 2), (2, 2)]:
        assert abs(oracle.wilson_loop(Uf, R, T) - oracle.wilson_loop(U, R, T)) < 1e-14
    assert oracle.unitarity_violation(Uf) < 1e-13
    h = r["history"][: r["iters"] + 1]
    assert np.all(np.diff(h[:, 1]) > -1e-6)  # float stage: F rises up to float roundoff
    # oracle values at the fixed links agree with the library's
    assert abs(oracle.theta(oracle.delta(Uf)) - r["theta"]) < 1e-16 + 1e-12 * r["theta"]
    assert abs(oracle.functional(Uf) - r["F"]) < 1e-12


def test_mixed_store_mid_float_stage_is_gauge_equivalent(lgf):
    dims = (8, 8, 4, 6)
    U = synth.config(dims, 9, 0.6)
    with lgf.Lattice(dims) as lat:
        lat.load(U, "mixed")
        r = lat.iterate(5, 0.08, 1e-15, theta_switch=1e-30)
        assert r["iters"] == 5
        Us = np.empty_like(U)
        lat.store(Us)
    assert abs(oracle.plaquette(Us) - oracle.plaquette(U)) < 1e-14
    assert oracle.unitarity_violation(Us) < 1e-13
    # the rebuilt links carry the float stage's progress
    th0 = oracle.theta(oracle.delta(U))
    assert oracle.theta(oracle.delta(Us)) < 0.5 * th0


def test_t_walking_kernels_match_site_order(lgf, monkeypatch):
    """Mixed fixes with the float and residual Delta and updates walking along t (8 slices per thread,
    forced at 16^4 with LGF_TWALK_MIN_BLOCKS=0) against the site-order kernels (LGF_TWALK=0): the same
    iterations, F to 1e-14 and the links to 1e-12 (theta, summed over other groups of sites, may decide a
    stage switch at another rounding)."""
    monkeypatch.setenv("LGF_TWALK_MIN_BLOCKS", "0")
    dims = (16, 16, 16, 16)
    U = synth.config(dims, 8, 0.6)
    res = []
    for flag in ("1", "0"):
        monkeypatch.setenv("LGF_TWALK", flag)
        Uf = U.copy()
        with lgf.Lattice(dims) as lat:
            r = lat.fix(Uf, 0.08, 1e-15, "mixed", max_iter=400)
        res.append((r, Uf))
    (r1, U1), (r0, U0) = res
    assert r1["converged"] and r0["converged"] and r1["iters"] == r0["iters"]
    assert abs(r1["F"] - r0["F"]) < 1e-14
    assert float(np.abs(U1 - U0).max()) < 1e-12


def test_mixed_float_stage_hands_over_when_theta_stalls(lgf):
    """A switch point below what float links resolve: the float stage stops lowering theta, hands over on
    its own, and the double stage converges with the links still gauge-equivalent to the input."""
    dims = (8, 8, 8, 8)
    U = synth.config(dims, 1, 0.3)
    with lgf.Lattice(dims) as lat:
        r = lat.fix(U.copy(), 0.08, 1e-15, "mixed", max_iter=1000, theta_switch=1e-30)
        Uf = U.copy()
        r = lat.fix(Uf, 0.08, 1e-15, "mixed", max_iter=1000, theta_switch=1e-30)
        r_ref = lat.fix(U.copy(), 0.08, 1e-15, "fp64")
    assert r["converged"] and r["theta"] < 1e-15
    assert r["iters"] < r_ref["iters"] + 40, (r, r_ref)
    assert abs(r["F"] - r_ref["F"]) < 1e-12
    assert abs(oracle.plaquette(Uf) - oracle.plaquette(U)) < 1e-14
    assert oracle.theta(oracle.delta(Uf)) < 1e-15


@pytest.mark.parametrize("split", ["00", "21", "44", "13"])
def test_handover_fixed_point_matches_fp64(lgf, monkeypatch, split):
    """The handover links G U0 G^+(x+mu) formed in 61-bit fixed point, or split between fixed point and FP64
    per direction (LGF_HANDOVER_SPLIT: FP64 directions in even and odd warps), agree with the FP64 product to
    a few units of the FP64 rounding, and all are gauge-equivalent to the input."""
    monkeypatch.setenv("LGF_HANDOVER_SPLIT", split)
    dims = (8, 8, 4, 6)
    U = synth.config(dims, 9, 0.6)

    def stored():
        with lgf.Lattice(dims) as lat:
            lat.load(U, "mixed")
            lat.iterate(7, 0.08, 1e-15, theta_switch=1e-30)
            out = np.empty_like(U)
            lat.store(out)
        return out
    Uq = stored()
    monkeypatch.setenv("LGF_HANDOVER_FP64", "1")
    Ud = stored()
    assert float(np.abs(Uq - Ud).max()) < 1e-15
    for Us in (Uq, Ud):
        assert abs(oracle.plaquette(Us) - oracle.plaquette(U)) < 1e-14
        assert oracle.unitarity_violation(Us) < 1e-13


def test_mixed_schedule_as_specified(lgf, monkeypatch):
    """The mixed schedule in its plainest form (float links, FFTs and updates with double reductions and a
    double-precision reprojection every 16 iterations until theta <= 1e-8, the handover, double iterations
    to theta < 1e-15): theta, F and the plaquette against the FP64 oracle and the double path."""
    monkeypatch.setenv("LGF_REUNIT_FP64", "1")
    monkeypatch.setenv("LGF_RESIDUAL", "0")
    dims = (16, 16, 16, 16)
    U = synth.config(dims, 7, 0.6)
    Um = U.copy()
    with lgf.Lattice(dims) as lat:
        lat.enable_timing(True)
        r = lat.fix(Um, 0.08, 1e-15, "mixed", theta_switch=1e-8)
        names = set(lat.kernel_times())
        r64 = lat.fix(U.copy(), 0.08, 1e-15, "fp64")
    assert "gauge_update.f64" in names and "update_residual.f32" not in names, names
    assert "gauge_update_fused_reunit.f32" in names
    assert r["converged"] and r["theta"] < 1e-15
    assert abs(r["F"] - r64["F"]) < 1e-12
    assert abs(r["iters"] - r64["iters"]) <= 3, (r["iters"], r64["iters"])
    assert oracle.theta(oracle.delta(Um)) < 1e-15
    assert abs(oracle.functional(Um) - r["F"]) < 1e-12
    assert abs(oracle.plaquette(Um) - oracle.plaquette(U)) < 1e-14


def test_fp32_precision_fix_reaches_float_floor(lgf):
    dims = (8, 8, 8, 8)
    U = synth.config(dims, 1, 0.3)
    with lgf.Lattice(dims) as lat:
        r = lat.fix(U.copy(), 0.08, 1e-9, "fp32", max_iter=500)
    assert r["converged"] and r["theta"] < 1e-9


def test_mixed_fft32_final_variant(lgf):
    """The double stage with a float Fourier filter: same fixed point, theta < 1e-15 in double, exact
    gauge equivalence, and the iteration count of the all-double final stage within a few."""
    dims = (16, 16, 16, 16)
    U = synth.config(dims, 7, 0.6)
    with lgf.Lattice(dims) as lat:
        r0 = lat.fix(U.copy(), 0.08, 1e-15, "mixed")
        Uf = U.copy()
        r1 = lat.fix(Uf, 0.08, 1e-15, "mixed", fft32_final=True)
        m = lat.measure(Uf)
    assert r1["converged"] and r1["theta"] < 1e-15 and m["theta"] < 1e-15
    assert abs(r1["iters"] - r0["iters"]) <= 3
    assert abs(r1["F"] - r0["F"]) < 1e-10
    assert abs(oracle.plaquette(Uf) - oracle.plaquette(U)) < 1e-14
