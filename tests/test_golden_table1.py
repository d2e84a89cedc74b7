"""Table 1 of the paper (tests/golden/table1_per_thread.txt) against the oracle's data dependencies.

The paper's per-thread load/store counts follow from which data each step reads per site. Here the oracle's
actual stencil footprints are found by brute force on a 3^4 lattice (perturb one input, see which outputs
move), and the counts Table 1 prints are rebuilt from them: a stencil that read other neighbours, or fewer or
more links, would not reproduce them. The FFT operation count convention of Sec. 2.2 is checked against the
bench's per-pass flop model."""
import math
import os
import sys

import numpy as np
import pytest

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))
DIMS = (3, 3, 3, 3)  # every +-mu neighbour of a site is distinct


def table1():
    rows = {}
    for line in open(os.path.join(HERE, "golden", "table1_per_thread.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, *v = line.split()
        rows[k] = tuple(int(x) for x in v)
    return rows


def site_index(t, z, y, x):
    return (t, z, y, x)


def test_delta_footprint_is_table1_k2():
    """Delta(x) (and theta, F partials) depends on exactly 8 links: 8 x 18 = 144 loads (18-real), 8 x 12 = 96
    (12-real); it stores the 9 complex entries of Delta plus the two partial sums: 20 (and 12 + 2 = 14)."""
    k2 = table1()["k2"]
    U = synth.config(DIMS, 31, 0.6)
    x = site_index(1, 1, 1, 1)
    D0 = oracle.delta(U)[x]
    touched = 0
    for idx in np.ndindex(U.shape[:5]):  # (mu, t, z, y, x)
        Up = U.copy()
        Up[idx] = Up[idx] @ np.diag([np.exp(0.01j), np.exp(-0.01j), 1.0])
        if np.abs(oracle.delta(Up)[x] - D0).max() > 1e-12:
            touched += 1
    assert touched == 8
    assert touched * 18 == k2[0] and touched * 12 == k2[3]
    assert 9 * 2 + 2 == k2[1] and 6 * 2 + 2 == k2[4]


def test_update_footprint_is_table1_k6():
    """The four new links of a site depend on the four old links and on g at 5 sites (x and its 4 forward
    neighbours): 9 matrices x 18 = 162 loads, 4 x 18 = 72 stores; 108 and 48 with 12 reals. The flop
    count is 8 SU(3) products of 27 complex multiplications and 18 complex additions each."""
    k6 = table1()["k6"]
    U = synth.config(DIMS, 32, 0.6)
    g = oracle.gauge_field(oracle.fourier_filter(oracle.delta(U)), 0.08)
    x = site_index(1, 1, 1, 1)
    base = oracle.gauge_transform(U, g)[:, 1, 1, 1, 1]
    g_sites = 0
    for idx in np.ndindex(g.shape[:4]):
        gp = g.copy()
        gp[idx] = gp[idx] @ np.diag([np.exp(0.01j), np.exp(-0.01j), 1.0])
        if np.abs(oracle.gauge_transform(U, gp)[:, 1, 1, 1, 1] - base).max() > 1e-12:
            g_sites += 1
    assert g_sites == 5
    assert (4 + g_sites) * 18 == k6[0] and (4 + g_sites) * 12 == k6[3]
    assert 4 * 18 == k6[1] and 4 * 12 == k6[4]
    assert 8 * (27 * 6 + 18 * 2) == k6[2]


def test_gauge_field_footprint_is_table1_k5():
    """g(x) depends on Delta-tilde(x) only: 18 loads and 18 stores (12 and 12 with 12 reals)."""
    k5 = table1()["k5"]
    U = synth.config(DIMS, 33, 0.6)
    Dt = oracle.fourier_filter(oracle.delta(U))
    g0 = oracle.gauge_field(Dt, 0.08)
    for idx in np.ndindex(Dt.shape[:4]):
        Dp = Dt.copy()
        Dp[idx] = Dp[idx] + 1e-3 * np.array([[0, 1, 0], [-1, 0, 0], [0, 0, 0]])
        d = np.abs(oracle.gauge_field(Dp, 0.08) - g0).max(axis=(-1, -2))
        assert np.argwhere(d > 1e-12).tolist() == [list(idx)]  # only g at the perturbed site moves
    assert 9 * 2 == k5[0] == k5[1] and 6 * 2 == k5[3] == k5[4]


@pytest.mark.parametrize("dims", [(64, 64, 64, 64), (32, 32, 32, 64)])
def test_fft_flop_convention_of_sec_2_2(dims):
    """The bench's FFT flop model of its five passes (xy forward, z forward, t forward + filter + inverse,
    z inverse, xy inverse) adds up to the paper's count nx ny nz nt 5 (log2(nx ny) + log2(nz nt)) per field
    and transform, for the 4 packed fields and 2 transforms (plus 6 flops per mode for the filter)."""
    sys.path.insert(0, os.path.dirname(HERE))
    import bench
    V = int(np.prod(dims))
    nx, ny, nz, nt = dims
    paper = V * 5 * (math.log2(nx * ny) + math.log2(nz * nt))
    total = sum(bench.work_model(k + ".f32", dims)[1]
                for k in ("fft_xy_fwd", "fft_z_fwd", "fft_t_filter", "fft_z_inv", "fft_xy_inv"))
    assert abs(total - (2 * 4 * paper + 4 * 6 * V)) <= 1e-9 * total
