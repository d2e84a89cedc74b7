"""Writes the oracle's complete gauge-fixing trajectories on the benchmarked configurations.

Each case runs Algorithm 1 (FP64 CPU oracle, alpha = 0.08) from a synthetic configuration until
theta < 1e-15 and stores, as JSON beside this script:
  - the (theta, F) pair of every iteration (Eq. 4 and Eq. 1 at g = 1, iteration 0 = the input),
  - the iteration count (gauge updates applied),
  - the average plaquette of the input and of the fixed links (gauge invariant; Sec. 1),
  - the largest deviation of the fixed links from unitarity,
  - the fixed links at a few sampled sites (all four directions).

Only `oracle/` and `synth/` are called: no expected value here comes from the CUDA library. The GPU
tests read these files and compare the library's trajectories with them.

Usage: python tests/golden/make_oracle_histories.py [case ...]   (default: every case; the 64^4 case
needs about 50 GB of host memory and runs for tens of minutes on 8 cores).
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402

ALPHA, EPS_STOP = 0.08, 1e-15


def ensemble_eps():
    """The ensemble's per-configuration roughness: eps_i ~ U[0.4, 0.7] from numpy seed 99, configuration i
    from seed 100 + i (16 each of 16^4, 24^3x48, 32^3x64, in that order)."""
    return np.random.default_rng(99).uniform(0.4, 0.7, 48)


def cases():
    e = ensemble_eps()
    return {
        "8x8x8x8_s1": ((8, 8, 8, 8), 1, 0.3),
        "32x32x32x32_s2": ((32, 32, 32, 32), 2, 0.6),
        "64x64x64x64_s4": ((64, 64, 64, 64), 4, 0.6),
        # one configuration of each ensemble shape: ensemble members 0, 16 and 32
        "16x16x16x16_s100": ((16, 16, 16, 16), 100, float(e[0])),
        "24x24x24x48_s116": ((24, 24, 24, 48), 116, float(e[16])),
        "32x32x32x64_s132": ((32, 32, 32, 64), 132, float(e[32])),
    }


def sample_sites(dims, n=8):
    """A fixed spread of sites (x, y, z, t): the corners of the lattice and a few interior points."""
    nx, ny, nz, nt = dims
    pts = [(0, 0, 0, 0), (nx - 1, ny - 1, nz - 1, nt - 1), (nx // 2, 1, nz - 2, nt // 3),
           (1, ny // 2, nz // 3, nt - 1), (nx // 3, ny // 3, nz // 2, nt // 2), (nx - 2, 0, 1, 2),
           (0, ny - 1, nz // 2, 1), (nx // 2, ny // 2, nz // 2, nt // 2)]
    return pts[:n]


def run_case(name, dims, seed, eps):
    t0 = time.time()
    U = synth.config(dims, seed, eps)
    plaq_in = oracle.plaquette(U)
    Uf, iters, th, F, hist = oracle.fix(U, ALPHA, EPS_STOP, 2000, hist_len=2001)
    del U
    sites = sample_sites(dims)
    links = {}
    for (x, y, z, t) in sites:
        m = Uf[:, t, z, y, x]  # (4, 3, 3)
        links["%d,%d,%d,%d" % (x, y, z, t)] = [[float(v.real), float(v.imag)] for v in m.reshape(-1)]
    out = {
        "what": "oracle (FP64 CPU) trajectory of Algorithm 1, alpha=%g, stop at theta < %g" % (ALPHA, EPS_STOP),
        "dims": list(dims), "seed": seed, "eps": eps, "generator": "synth.config, Haar h, algebra norm 1/(2 sqrt 2)",
        "alpha": ALPHA, "eps_stop": EPS_STOP, "iters": int(iters), "theta": th, "F": F,
        "history": [[float(a), float(b)] for a, b in hist],
        "plaquette_in": plaq_in, "plaquette_out": oracle.plaquette(Uf),
        "unitarity_violation_out": oracle.unitarity_violation(Uf),
        "links_out_at_sites": links,
        "links_layout": "per site: 4 directions x 3 x 3 row-major complex entries as [re, im]",
        "oracle_seconds": round(time.time() - t0, 1), "host_threads": os.cpu_count(),
    }
    path = os.path.join(HERE, "oracle_fix_%s.json" % name)
    with open(path + ".tmp", "w") as f:
        json.dump(out, f, indent=1)
    os.replace(path + ".tmp", path)
    print("%s: %d iterations, theta %.3e, F %.16f, %.0f s" % (name, iters, th, F, out["oracle_seconds"]), flush=True)


def main():
    todo = cases()
    names = sys.argv[1:] or list(todo)
    for n in names:
        run_case(n, *todo[n])


if __name__ == "__main__":
    main()
