"""Whole gauge fixings at the benchmarked sizes against the oracle's complete trajectories.

The oracle (FP64 CPU, Algorithm 1) was run to theta < 1e-15 on each configuration by
tests/golden/make_oracle_histories.py, which calls only the oracle and the input generator; the JSON
files beside it hold every iteration's theta (Eq. 4) and F (Eq. 1 at g = 1), the iteration count, the
plaquette of the input and of the fixed links, and the fixed links at a few sites.

Checked here, through the C ABI:
  - the double path, with its Fourier filter in double-float (the default) and in IEEE double: theta and F
    of every iteration (theta within 1e-12 relative plus the roundoff floor 64 u_f sqrt(theta) of the
    filter's arithmetic, F within 1e-12 relative), the iteration count within +-1, the fixed links at the
    sampled sites, and the plaquette;
  - the mixed schedule as the library runs it by default, and the mixed schedule as specified (float to
    theta <= 1e-8 with double reprojection, then double iterations): theta < 1e-15, the final F within
    1e-12 of the oracle's, the iteration count within +-1, the plaquette of the input kept;
  - an ensemble holding one configuration of each shape of the benchmarked ensemble (16^4, 24^3x48,
    32^3x64, the first shape twice), in the double path and in the mixed schedule.
The first entry of the double path's history is the input's theta and F, so the input that the generator
produced on this machine is checked against the one the oracle fixed."""
import contextlib
import json
import os

import numpy as np
import pytest

import synth
from gpu_common import theta_tol

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
SINGLE = ["8x8x8x8_s1", "32x32x32x32_s2", "64x64x64x64_s4"]
ENSEMBLE = ["16x16x16x16_s100", "24x24x24x48_s116", "32x32x32x64_s132", "16x16x16x16_s100"]

# Fixed links at the sampled sites. Double path with the oracle's iteration count: the trajectories agree
# step by step at FP64 rounding, so the links agree to 1e-11. Otherwise (one iteration apart, or another
# schedule) both results lie within the convergence radius of the same maximum: at theta < 1e-15 the
# per-site |Delta| is below ~6e-8, and the remaining gauge rotation, Delta divided by the smallest
# nonzero p^2 of the lattice (4 sin^2(pi/64) = 9.6e-3 at 64^4), is below ~1e-5.
LINKS_SAME_TRAJECTORY = 1e-11
LINKS_SAME_MAXIMUM = 1e-5


def golden(name):
    with open(os.path.join(GOLDEN, "oracle_fix_%s.json" % name)) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def lgf():
    import torch
    assert torch.cuda.is_available()
    import paper_1210_8018_gb300 as m
    return m


@contextlib.contextmanager
def env(**kv):
    saved = {k: os.environ.get(k) for k in kv}
    os.environ.update({k: str(v) for k, v in kv.items()})
    try:
        yield
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def links_at_sites(Ud, g):
    out = {}
    for key in g["links_out_at_sites"]:
        x, y, z, t = (int(v) for v in key.split(","))
        out[key] = Ud[:, t, z, y, x].cpu().numpy().reshape(-1)
    return out


def check_links(Ud, g, tol):
    got = links_at_sites(Ud, g)
    worst = 0.0
    for key, ref in g["links_out_at_sites"].items():
        r = np.array([complex(a, b) for a, b in ref])
        worst = max(worst, float(np.abs(got[key] - r).max()))
    assert worst <= tol, "sampled links differ by %.3e > %.1e" % (worst, tol)
    return worst


def check_input(h0, g):
    """Iteration 0 is the input: the generator made the same configuration here."""
    th0, F0 = g["history"][0]
    assert abs(h0[1] - F0) <= 1e-12 * abs(F0), (h0, g["history"][0])
    assert abs(h0[0] - th0) <= theta_tol(th0), (h0, g["history"][0])


def check_final(r, plaq, g):
    assert r["theta"] < 1e-15, r
    assert abs(r["iters"] - g["iters"]) <= 1, (r["iters"], g["iters"])
    assert abs(r["F"] - g["F"]) <= 1e-12 * abs(g["F"]), (r["F"], g["F"])
    assert abs(plaq - g["plaquette_in"]) <= 1e-13, (plaq, g["plaquette_in"])
    assert abs(plaq - g["plaquette_out"]) <= 1e-13, (plaq, g["plaquette_out"])


def dev_config(g):
    import torch
    U = synth.config(tuple(g["dims"]), g["seed"], g["eps"])
    return torch.from_numpy(U).to("cuda")


# The unit roundoff of the arithmetic that sets each step's direction: the Fourier filter of the double path
# runs in double-float (two floats, a 48-bit significand) by default, or in IEEE double
# (LGF_FFT_NATIVE_F64=1). Along a whole trajectory the two implementations (oracle and library) drift apart
# by the rounding of that filter, accumulated over the iterations: theta is compared with the tolerance of
# a single evaluation, 1e-12 theta + 64 u_f sqrt(theta), u_f being that unit roundoff (2^-53 for IEEE
# double; 2^-48 for double-float). F (1e-12 relative) does not depend on the filter's precision.
FILTERS = {"double-float": ({}, 2.0 ** -48), "ieee-double": ({"LGF_FFT_NATIVE_F64": 1}, 2.0 ** -53)}


def theta_tol_filter(theta_ref, u_f):
    return 1e-12 * theta_ref + 64 * u_f * np.sqrt(theta_ref)


@pytest.mark.parametrize("filt", sorted(FILTERS))
@pytest.mark.parametrize("name", SINGLE)
def test_double_path_whole_trajectory(lgf, name, filt):
    switches, u_f = FILTERS[filt]
    g = golden(name)
    Ud = dev_config(g)
    with env(**switches):
        lat = lgf.Lattice(tuple(g["dims"]))  # the switches are read when the context is created
    with lat:
        r = lat.fix(Ud, g["alpha"], g["eps_stop"], "fp64", history_len=len(g["history"]) + 8)
        plaq = lat.measure(Ud)["plaquette"]
    h, ho = r["history"], np.array(g["history"])
    check_input(h[0], g)
    n = min(len(h), len(ho))
    for k in range(n):
        assert abs(h[k, 1] - ho[k, 1]) <= 1e-12 * abs(ho[k, 1]), (k, h[k], ho[k])
        assert abs(h[k, 0] - ho[k, 0]) <= theta_tol_filter(ho[k, 0], u_f), (k, h[k], ho[k])
    check_final(r, plaq, g)
    check_links(Ud, g, LINKS_SAME_TRAJECTORY if r["iters"] == g["iters"] else LINKS_SAME_MAXIMUM)


@pytest.mark.parametrize("name", SINGLE)
def test_mixed_default_against_oracle(lgf, name):
    g = golden(name)
    Ud = dev_config(g)
    with lgf.Lattice(tuple(g["dims"])) as lat:
        r = lat.fix(Ud, g["alpha"], g["eps_stop"], "mixed")
        plaq = lat.measure(Ud)["plaquette"]
    check_final(r, plaq, g)
    check_links(Ud, g, LINKS_SAME_MAXIMUM)


@pytest.mark.parametrize("name", SINGLE)
def test_mixed_as_specified_against_oracle(lgf, name):
    """Float links, FFTs and updates with double reductions and a double reprojection every 16 iterations
    until theta <= 1e-8; the double handover; double iterations to theta < 1e-15."""
    g = golden(name)
    Ud = dev_config(g)
    with env(LGF_REUNIT_FP64=1, LGF_RESIDUAL=0):
        lat = lgf.Lattice(tuple(g["dims"]))  # the switches are read when the context is created
    with lat:
        r = lat.fix(Ud, g["alpha"], g["eps_stop"], "mixed", theta_switch=1e-8)
        plaq = lat.measure(Ud)["plaquette"]
    check_final(r, plaq, g)
    check_links(Ud, g, LINKS_SAME_MAXIMUM)


@pytest.fixture(scope="module")
def tune_cache(tmp_path_factory):
    path = str(tmp_path_factory.mktemp("tune") / "fft_tune.json")
    with env(LGF_TUNE_CACHE=path):
        yield path


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_ensemble_of_the_benchmarked_shapes(lgf, tune_cache, precision):
    """One ensemble of 16^4, 24^3x48, 32^3x64 and 16^4 again (the shapes whose FFT passes the tuner picks
    among the radix-3, 48- and 64-long specialised and the generic passes), every member against the
    oracle's whole fix of that configuration."""
    gs = [golden(n) for n in ENSEMBLE]
    Us = [dev_config(g) for g in gs]
    with env(LGF_TUNE_CACHE=tune_cache):
        with lgf.Batch([tuple(g["dims"]) for g in gs]) as b:
            res = b.fix(Us, 0.08, 1e-15, precision)
            info = b.describe()
    assert len(info["groups"]) == 3 and info["graph_replays"] > 0
    for U, g, r in zip(Us, gs, res):
        assert r["status"] == lgf.LGF_OK, r
        with lgf.Lattice(tuple(g["dims"])) as lat:
            plaq = lat.measure(U)["plaquette"]
        check_final(r, plaq, g)
        if precision == "fp64":
            check_links(U, g, LINKS_SAME_TRAJECTORY if r["iters"] == g["iters"] else LINKS_SAME_MAXIMUM)
        else:
            check_links(U, g, LINKS_SAME_MAXIMUM)
