"""The gauge functional as a differentiable function of omega(x) in su(3), g = exp(i omega):
forward against the oracle's F_U[g] (Eq. 1) with g from scipy's matrix exponential; the hand-written
backward against the oracle's Delta at omega = 0 (dF/d omega^a = -(i/(24V)) Tr[T^a Delta]) and against
central finite differences (h = 1e-6) at omega ~ N(0, 0.05^2) per generator; torch.autograd.gradcheck;
and Adam on omega driving theta of the transformed links down."""
import numpy as np
import pytest
import scipy.linalg

import oracle
import synth
from helpers import gell_mann

pytestmark = pytest.mark.gpu
T = gell_mann() / 2


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available()
    import paper_1210_8018_gb300 as lgf
    return torch, lgf


def omega_field(dims, seed, sigma):
    V = int(np.prod(dims))
    return synth.normals(seed, 0, V * 8, sigma).reshape(V, 8)


def expm_field(omega, dims):
    nx, ny, nz, nt = dims
    H = np.einsum("sa,aij->sij", omega, T)
    g = np.stack([scipy.linalg.expm(1j * h) for h in H])
    return np.ascontiguousarray(g.reshape(nt, nz, ny, nx, 3, 3))


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (24, 24, 24, 24)])
def test_forward_matches_oracle(env, dims):
    torch, lgf = env
    U = synth.config(dims, 5, 0.5)
    om = omega_field(dims, 6, 0.05)
    g_ref = expm_field(om, dims)
    F_ref = oracle.functional(U, g_ref)
    with lgf.Lattice(dims) as lat:
        g = np.empty_like(g_ref)
        F = lat.functional(U, om, g)
    np.testing.assert_allclose(g, g_ref, rtol=0, atol=2e-14)
    assert abs(F - F_ref) <= 1e-12 * abs(F_ref)


@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (24, 24, 24, 24)])
def test_gradient_at_zero_is_delta(env, dims):
    torch, lgf = env
    V = int(np.prod(dims))
    U = synth.config(dims, 5, 0.5)
    D = oracle.delta(U).reshape(V, 3, 3)
    ref = (-1j / (24 * V) * np.einsum("aij,sji->sa", T, D)).real
    with lgf.Lattice(dims) as lat:
        grad = np.empty((V, 8))
        lat.functional_grad(U, np.zeros((V, 8)), grad)
    scale = np.abs(ref).max()
    assert np.abs(grad - ref).max() <= 1e-12 * scale


def local_F(U, g, y, dims):
    """12V times the part of F_U[g] (Eq. 1) that involves g(y): the 8 links that touch site y."""
    nx, ny, nz, nt = dims
    t, z, yy, x = y
    tot = 0.0
    for mu, (dt, dz, dy, dx) in enumerate([(0, 0, 0, 1), (0, 0, 1, 0), (0, 1, 0, 0), (1, 0, 0, 0)]):
        fw = ((t + dt) % nt, (z + dz) % nz, (yy + dy) % ny, (x + dx) % nx)
        bw = ((t - dt) % nt, (z - dz) % nz, (yy - dy) % ny, (x - dx) % nx)
        tot += np.trace(g[y] @ U[(mu,) + y] @ g[fw].conj().T).real
        tot += np.trace(g[bw] @ U[(mu,) + bw] @ g[y].conj().T).real
    return tot


def test_gradient_finite_differences(env):
    torch, lgf = env
    dims = (24, 24, 24, 24)
    V = int(np.prod(dims))
    U = synth.config(dims, 5, 0.5)
    om = omega_field(dims, 6, 0.05)
    with lgf.Lattice(dims) as lat:
        grad = np.empty((V, 8))
        lat.functional_grad(U, om, grad)
    g = expm_field(om, dims)
    rng = np.random.default_rng(0)
    h = 1e-6
    nx, ny, nz, nt = dims
    for _ in range(6):
        s = int(rng.integers(0, V))
        y = (s // (nx * ny * nz), (s // (nx * ny)) % nz, (s // nx) % ny, s % nx)
        for a in range(8):
            vals = []
            for sgn in (1, -1):
                w = om[s].copy()
                w[a] += sgn * h
                gp = g.copy()
                gp[y] = scipy.linalg.expm(1j * np.einsum("a,aij->ij", w, T))
                vals.append(local_F(U, gp, y, dims))
            fd = (vals[0] - vals[1]) / (2 * h)  # = 12 V dF/d omega^a
            assert abs(12 * V * grad[s, a] - fd) < 2e-8, (s, a, 12 * V * grad[s, a], fd)


def test_autograd_function_and_gradcheck(env):
    torch, lgf = env
    dims = (2, 2, 2, 2)
    U = torch.from_numpy(synth.config(dims, 7, 0.5)).cuda()
    om = torch.from_numpy(omega_field(dims, 8, 0.05)).cuda().requires_grad_(True)
    LandauF = lgf.LandauF()
    with lgf.Lattice(dims) as lat:
        F = LandauF.apply(om, U, lat)
        F.backward()
        g2 = torch.empty_like(om)
        lat.functional_grad(U, om.detach(), g2)
        assert torch.equal(om.grad, g2)
        assert torch.autograd.gradcheck(lambda w: LandauF.apply(w, U, lat), (om.detach().requires_grad_(True),),
                                        eps=1e-6, atol=1e-8, rtol=1e-5)


def test_adam_drives_theta_down(env):
    torch, lgf = env
    dims = (8, 8, 8, 8)
    U = synth.config(dims, 1, 0.3, h_mode=synth.H_NEAR_IDENTITY, h_scale=0.3)
    res = lgf.adam_fix(torch.from_numpy(U).cuda(), target=1e-10, max_steps=4000)
    assert res["theta"] <= 1e-10, res
    assert res["F"] > res["F0"]


def test_sgd_on_preconditioned_gradient_reproduces_algorithm_1(env):
    """torch.optim.SGD on the Fourier-preconditioned gradient with lr = 24 alpha V and re-basing after
    each step is Algorithm 1's step (exponential instead of first order): it converges like the
    library's own fix."""
    torch, lgf = env
    dims = (8, 8, 8, 8)
    V = 8 ** 4
    U = synth.config(dims, 1, 0.3)
    with lgf.Lattice(dims) as lat:
        r_ref = lat.fix(U.copy(), 0.08, 1e-10, "fp64")
    res = lgf.adam_fix(torch.from_numpy(U).cuda(), target=1e-10, optimizer="sgd", precondition=True,
                       lr=24 * 0.08 * V, rebase_every=1, check_every=1, max_steps=200)
    assert res["theta"] <= 1e-10
    assert abs(res["steps"] - r_ref["iters"]) <= 3, (res["steps"], r_ref["iters"])
    assert abs(res["F"] - r_ref["F"]) < 1e-8
