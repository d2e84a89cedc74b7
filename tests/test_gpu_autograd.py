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
    """torch.optim.SGD on the Fourier-preconditioned gradient with lr = alpha (the loss is -24 V F) and
    re-basing after each step is Algorithm 1's step (exponential instead of first order): it converges like the
    library's own fix."""
    torch, lgf = env
    dims = (8, 8, 8, 8)
    U = synth.config(dims, 1, 0.3)
    with lgf.Lattice(dims) as lat:
        r_ref = lat.fix(U.copy(), 0.08, 1e-10, "fp64")
    res = lgf.adam_fix(torch.from_numpy(U).cuda(), target=1e-10, optimizer="sgd", precondition=True,
                       lr=0.08, rebase_every=1, check_every=1, max_steps=200)
    assert res["theta"] <= 1e-10
    assert abs(res["steps"] - r_ref["iters"]) <= 3, (res["steps"], r_ref["iters"])
    assert abs(res["F"] - r_ref["F"]) < 1e-8


@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (6, 4, 8, 10), (24, 24, 24, 24)])
def test_filter_on_coefficients_matches_oracle_matrix_filter(env, dims):
    """lgf_filter_coeffs on the eight coefficient fields equals the oracle's filter of the matrix field
    i sum_a c^a T^a, element by element, read back in coefficients (c^a = 2 Tr[T^a (-i M)])."""
    torch, lgf = env
    V = int(np.prod(dims))
    nx, ny, nz, nt = dims
    c = synth.normals(11, 0, V * 8, 0.3).reshape(V, 8)
    M = 1j * np.einsum("sa,aij->sij", c, T).reshape(nt, nz, ny, nx, 3, 3)
    Mt = oracle.fourier_filter(np.ascontiguousarray(M)).reshape(V, 3, 3)
    ref = 2 * np.einsum("aij,sji->sa", T, -1j * Mt).real
    with lgf.Lattice(dims) as lat:
        out = np.empty_like(c)
        lat.filter_coeffs(c, out)
        cd = torch.from_numpy(c).cuda()
        lat.filter_coeffs(cd, cd)  # in place, device pointers
    scale = np.abs(ref).max()
    assert np.abs(out - ref).max() <= 1e-12 * scale
    assert np.abs(cd.cpu().numpy() - ref).max() <= 1e-12 * scale


def test_adam_on_preconditioned_gradient_reaches_1e_10_on_the_rough_field(env):
    """The differentiation workload: 24^4, eps = 0.5, omega ~ N(0, 0.05^2) per generator. torch.optim.Adam
    on the Fourier-preconditioned gradient (lgf_filter_coeffs), with omega re-based into the links every 5
    steps and Adam's moments carried across re-basings, reaches theta <= 1e-10 at the maximum that
    Algorithm 1 finds from the same links. (Plain Adam on this field slows down critically.)"""
    torch, lgf = env
    dims = (24, 24, 24, 24)
    U = synth.config(dims, 5, 0.5)
    om = torch.from_numpy(omega_field(dims, 6, 0.05)).cuda()
    with lgf.Lattice(dims) as lat:
        r_ref = lat.fix(U.copy(), 0.08, 1e-12, "fp64")
    Ud = torch.from_numpy(U).cuda()
    res = lgf.adam_fix(Ud, target=1e-10, omega0=om, lr=0.05, precondition=True, rebase_every=5, check_every=5,
                       patience=2, max_steps=2000)
    assert res["theta"] <= 1e-10, res["theta"]
    assert res["steps"] < 2000
    assert abs(res["F"] - r_ref["F"]) <= 1e-9, (res["F"], r_ref["F"])
    with lgf.Lattice(dims) as lat:
        m = lat.measure(Ud)
    assert m["theta"] <= 1e-10 and abs(m["F"] - res["F"]) <= 1e-14
    assert abs(m["plaquette"] - oracle.plaquette(U)) < 1e-13
