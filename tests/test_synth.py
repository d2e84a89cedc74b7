"""Checks of the seeded configuration generator (inputs only)."""
import numpy as np

import oracle
import synth


def test_links_su3_and_deterministic():
    U = synth.config((4, 4, 4, 4), 1, 0.6)
    assert oracle.unitarity_violation(U) < 1e-14
    assert np.array_equal(U, synth.config((4, 4, 4, 4), 1, 0.6))
    assert not np.array_equal(U, synth.config((4, 4, 4, 4), 2, 0.6))


def test_plaquette_targets():
    # eps = 0.6 gives an average plaquette in the 0.55-0.65 window of the rough ensemble
    assert 0.55 < oracle.plaquette(synth.config((8, 8, 8, 8), 2, 0.6)) < 0.65
    # pure gauge: plaquette 1
    assert abs(oracle.plaquette(synth.config((4, 4, 4, 4), 3, 0.0)) - 1) < 1e-14


def test_haar_moments():
    """Links of a pure-gauge Haar field are Haar distributed: E[Tr U] = 0, E|Tr U|^2 = 1."""
    U = synth.config((8, 8, 8, 8), 5, 0.0)
    tr = np.trace(U, axis1=-2, axis2=-1).ravel()
    n = tr.size
    assert abs(tr.mean()) < 5 / np.sqrt(n)
    assert abs(np.mean(abs(tr) ** 2) - 1) < 8 / np.sqrt(n)


def test_normals_moments():
    z = synth.normals(3, 0, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01
    w = synth.normals(3, 1, 200000)
    assert abs(np.corrcoef(z, w)[0, 1]) < 0.01
