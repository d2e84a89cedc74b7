"""Ensembles of uneven lattice shapes fixed together (grouped launches, CUDA-graph replay, autotuned
FFT passes): every configuration against the FP64 oracle, per-configuration iteration counts and
statuses, and the mixed schedule's exact gauge equivalence."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import assert_matrix_close

pytestmark = pytest.mark.gpu

SHAPES = [(8, 8, 8, 8), (6, 4, 8, 10), (8, 8, 8, 8), (16, 16, 8, 8), (6, 4, 8, 10)]
EPS = [0.4, 0.55, 0.7, 0.5, 0.45]


@pytest.fixture(scope="module")
def lgf(tmp_path_factory):
    import os
    import torch
    assert torch.cuda.is_available()
    os.environ["LGF_TUNE_CACHE"] = str(tmp_path_factory.mktemp("tune") / "fft_tune.json")
    import paper_1210_8018_gb300 as m
    return m


def configs():
    return [synth.config(d, 100 + i, e) for i, (d, e) in enumerate(zip(SHAPES, EPS))]


def test_batch_fp64_matches_oracle(lgf):
    import torch
    Us = configs()
    Ud = [torch.from_numpy(U.copy()).cuda() for U in Us]
    with lgf.Batch(SHAPES) as b:
        res = b.fix(Ud, 0.08, 1e-15, "fp64")
        info = b.describe()
    assert len(info["groups"]) == 3 and info["graph_replays"] > 0
    for U, Uf, r in zip(Us, Ud, res):
        Uo, it, th, F, _ = oracle.fix(U, 0.08, 1e-15, 2000)
        assert r["status"] == lgf.LGF_OK and r["theta"] < 1e-15
        assert abs(r["iters"] - it) <= 1, (r, it)
        assert abs(r["F"] - F) <= 1e-12 * abs(F)
        assert_matrix_close(Uf.cpu().numpy(), Uo, rtol=1e-11)


def test_batch_mixed_and_host_buffers(lgf):
    Us = configs()
    work = [U.copy() for U in Us]
    with lgf.Batch(SHAPES) as b:
        res = b.fix(work, 0.08, 1e-15, "mixed")
    for U, Uf, r in zip(Us, work, res):
        assert r["status"] == lgf.LGF_OK and r["theta"] < 1e-15
        assert abs(oracle.plaquette(Uf) - oracle.plaquette(U)) < 1e-14
        assert oracle.unitarity_violation(Uf) < 1e-13
        assert oracle.theta(oracle.delta(Uf)) < 1e-15


def test_batch_limits_and_repeat(lgf):
    Us = configs()
    with lgf.Batch(SHAPES) as b:
        res = b.fix([U.copy() for U in Us], 0.08, 1e-15, "fp64", max_iter=4)
        assert all(r["iters"] == 4 and r["status"] == lgf.LGF_ENOCONV for r in res)
        # the same batch object again (graph reused) gives the single-context results
        res2 = b.fix([U.copy() for U in Us], 0.08, 1e-15, "fp64")
    for U, r in zip(Us, res2):
        with lgf.Lattice(oracle.dims_of_links(U)) as lat:
            r1 = lat.fix(U.copy(), 0.08, 1e-15, "fp64")
        assert abs(r1["iters"] - r["iters"]) <= 1 and abs(r1["F"] - r["F"]) <= 1e-12 * abs(r1["F"])


def test_batch_mixed_float_stage_hands_over_when_theta_stalls(lgf):
    Us = configs()
    work = [U.copy() for U in Us]
    with lgf.Batch(SHAPES) as b:
        res = b.fix(work, 0.08, 1e-15, "mixed", max_iter=1000, theta_switch=1e-30)
    for U, Uf, r in zip(Us, work, res):
        assert r["status"] == lgf.LGF_OK and r["theta"] < 1e-15 and r["iters"] < 1000
        assert abs(oracle.plaquette(Uf) - oracle.plaquette(U)) < 1e-14
        assert oracle.theta(oracle.delta(Uf)) < 1e-15


def test_batch_mixed_matches_single_contexts(lgf):
    """The ensemble's mixed schedule (float stage, handover, residual stage, rebuild) gives each configuration
    the fixed point and, within the replay granularity, the iteration count of a single-context fix."""
    Us = configs()
    with lgf.Batch(SHAPES) as b:
        res = b.fix([U.copy() for U in Us], 0.08, 1e-15, "mixed")
    for U, r in zip(Us, res):
        with lgf.Lattice(oracle.dims_of_links(U)) as lat:
            r1 = lat.fix(U.copy(), 0.08, 1e-15, "mixed")
        assert r["status"] == lgf.LGF_OK and r1["converged"] and r["theta"] < 1e-15
        assert abs(r1["iters"] - r["iters"]) <= 2, (r, r1)
        assert abs(r1["F"] - r["F"]) <= 1e-12 * abs(r1["F"])
