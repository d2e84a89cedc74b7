"""Parity at the full sizes of the benchmarked workloads.

32^4 (eps = 0.6, seed 2; and pure gauge): the oracle runs a few iterations of Algorithm 1 in seconds,
so the first iterations are compared element by element, plus one-step parity from a mid-trajectory
GPU state. 64^4 (eps = 0.6, seed 4, the mixed schedule the benchmark times, and the double path): the
oracle is too slow for a whole trajectory, so it runs the first two iterations and one iteration from the
mixed schedule's handover state; the fixed links are checked through quantities it computes in one pass
(theta, F, plaquette, unitarity), and the Fourier filter through the identity -d^2 (filtered Delta) =
p^2_max Delta at sampled sites, which holds at any size."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import assert_matrix_close, theta_tol

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


def test_32_4_fp64_first_iterations_and_one_step(lgf):
    dims = (32, 32, 32, 32)
    U = synth.config(dims, 2, 0.6)
    _, _, _, _, h_o = oracle.fix(U, 0.08, 0.0, 2, hist_len=3)
    Ud = dev(U)
    with lgf.Lattice(dims) as lat:
        r = lat.fix(Ud, 0.08, 1e-15, "fp64", history_len=200)
        assert r["converged"] and r["theta"] < 1e-15
        for k in range(3):
            assert abs(r["history"][k, 1] - h_o[k, 1]) <= 1e-12 * abs(h_o[k, 1])
            assert abs(r["history"][k, 0] - h_o[k, 0]) <= theta_tol(h_o[k, 0])
        # one-step parity from the GPU state after 10 iterations
        lat.load(dev(U), "fp64")
        lat.iterate(10, 0.08, 0.0)
        Uk = np.empty_like(U)
        lat.store(Uk)
        lat.load(Uk, "fp64")
        r1 = lat.iterate(1, 0.08, 0.0)
        U1 = np.empty_like(U)
        lat.store(U1)
    Uo, _, th_o, F_o, _ = oracle.fix(Uk, 0.08, 0.0, 1, hist_len=2)
    assert_matrix_close(U1, Uo)
    assert abs(r1["F"] - F_o) <= 1e-12 * abs(F_o)
    assert abs(r1["theta"] - th_o) <= theta_tol(th_o)
    Uf = Ud.cpu().numpy()
    assert abs(oracle.plaquette(Uf) - oracle.plaquette(U)) < 1e-14
    assert oracle.unitarity_violation(Uf) < 1e-13


def test_32_4_pure_gauge(lgf):
    dims = (32, 32, 32, 32)
    with lgf.Lattice(dims) as lat:
        U = synth.config(dims, 3, 0.0, h_mode=synth.H_NEAR_IDENTITY, h_scale=0.5)
        r = lat.fix(dev(U), 0.08, 1e-15, "fp64")
        assert r["converged"] and abs(r["F"] - 1) < 1e-12
        U = synth.config(dims, 3, 0.0)  # Haar gauge rotation: theta < eps, F <= 1 (possibly a Gribov copy)
        r = lat.fix(dev(U), 0.08, 1e-15, "mixed")
        assert r["converged"] and r["F"] <= 1 + 1e-14


def test_64_4_mixed_fix_invariants(lgf):
    dims = (64, 64, 64, 64)
    U = synth.config(dims, 4, 0.6)
    plaq0 = oracle.plaquette(U)
    Ud = dev(U)
    with lgf.Lattice(dims) as lat:
        r = lat.fix(Ud, 0.08, 1e-15, "mixed")
    assert r["converged"] and r["theta"] < 1e-15
    Uf = Ud.cpu().numpy()
    del Ud
    D = oracle.delta(Uf)
    th = oracle.theta(D)
    del D
    assert th < 1e-15 and abs(th - r["theta"]) <= theta_tol(r["theta"])
    F = oracle.functional(Uf)
    assert abs(F - r["F"]) <= 1e-12 * abs(F)
    assert abs(oracle.plaquette(Uf) - plaq0) < 1e-14
    assert oracle.unitarity_violation(Uf) < 1e-13


def test_64_4_double_path_invariants_and_same_maximum(lgf):
    """The double path at full size (its small-step forms run on every warp of the later iterations):
    the oracle's theta, F, plaquette and unitarity of the fixed links; and the mixed schedule reaches the
    same maximum of F on this field."""
    dims = (64, 64, 64, 64)
    U = synth.config(dims, 4, 0.6)
    plaq0 = oracle.plaquette(U)
    Ud = dev(U)
    with lgf.Lattice(dims) as lat:
        r = lat.fix(Ud, 0.08, 1e-15, "fp64")
        Um = dev(U)
        del U
        rm = lat.fix(Um, 0.08, 1e-15, "mixed")
        del Um
    assert r["converged"] and r["theta"] < 1e-15
    assert rm["converged"] and abs(rm["F"] - r["F"]) <= 1e-12 * abs(r["F"])
    Uf = Ud.cpu().numpy()
    del Ud
    D = oracle.delta(Uf)
    th = oracle.theta(D)
    del D
    assert th < 1e-15 and abs(th - r["theta"]) <= theta_tol(r["theta"])
    F = oracle.functional(Uf)
    assert abs(F - r["F"]) <= 1e-12 * abs(F)
    assert abs(oracle.plaquette(Uf) - plaq0) < 1e-14
    assert oracle.unitarity_violation(Uf) < 1e-13


def test_64_4_first_iterations_and_one_step_from_the_handover(lgf):
    """At the benchmarked size and configuration: theta and F of the first two double-path iterations
    against the oracle's; and one double-path iteration, element by element, from the mixed schedule's
    state at the handover (theta <= 1e-8, where its double stage starts and every warp takes the small-step
    forms)."""
    dims = (64, 64, 64, 64)
    U = synth.config(dims, 4, 0.6)
    _, _, _, _, h_o = oracle.fix(U, 0.08, 0.0, 2, hist_len=3)
    with lgf.Lattice(dims) as lat:
        lat.load(U, "fp64")
        r = lat.iterate(2, 0.08, 0.0, history_len=3)
        for k in range(3):
            assert abs(r["history"][k, 1] - h_o[k, 1]) <= 1e-12 * abs(h_o[k, 1]), (k, r["history"][k], h_o[k])
            assert abs(r["history"][k, 0] - h_o[k, 0]) <= theta_tol(h_o[k, 0]), (k, r["history"][k], h_o[k])
        lat.load(U, "mixed")
        rh = lat.iterate(1 << 30, 0.08, 1e-8)  # stops at the handover: theta < 1e-8 in the double stage
        assert rh["theta"] < 1e-8
        del U
        Uh = np.empty(synth.links_shape(dims), dtype=np.complex128)
        lat.store(Uh)
        lat.load(Uh, "fp64")
        r1 = lat.iterate(1, 0.08, 0.0)
        U1 = np.empty_like(Uh)
        lat.store(U1)
    Uo, _, th_o, F_o, _ = oracle.fix(Uh, 0.08, 0.0, 1, hist_len=2)
    del Uh
    assert_matrix_close(U1, Uo)
    assert abs(r1["F"] - F_o) <= 1e-12 * abs(F_o)
    assert abs(r1["theta"] - th_o) <= theta_tol(th_o)


def test_64_4_filter_laplacian_identity_sampled(lgf):
    """Delta-tilde = F^-1[(p2max/p2) F Delta]/V satisfies sum_mu [2 Dt(x) - Dt(x+mu) - Dt(x-mu)] = p2max Delta(x)
    (sum_x Delta = 0): checked at sampled sites for the double (df64) and the float filter."""
    dims = (64, 64, 64, 64)
    U = synth.config(dims, 4, 0.6)
    with lgf.Lattice(dims) as lat:
        D = np.empty(U.shape[1:], dtype=np.complex128)
        lat.delta(U, D)
        del U
        for prec, rtol in (("fp64", 1e-12), ("fp32", 2e-5)):
            Dt = np.empty_like(D)
            lat.filter(D, Dt, prec)
            scale = float(np.abs(Dt).max())
            rng = np.random.default_rng(1)
            for _ in range(40):
                x = tuple(int(rng.integers(0, 64)) for _ in range(4))  # (t, z, y, x)
                lap = 8 * Dt[x]
                for ax in range(4):
                    for d in (1, -1):
                        y = list(x)
                        y[ax] = (y[ax] + d) % 64
                        lap = lap - Dt[tuple(y)]
                assert np.abs(lap - 16.0 * D[x]).max() <= rtol * 16 * scale, (prec, x)
