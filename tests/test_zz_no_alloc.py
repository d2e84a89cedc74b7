"""lgf_delta_noalloc: the measurement entry point that allocates nothing, for callers that cannot call
cudaMalloc when they need theta, F and Delta (a framework pool that owns all device memory, a loop
that must not stall on an allocation, an out-of-memory handler). Its output must match the regular
lgf_delta entry point within the tolerances of the other parity tests, on two calls in a row (the
second call reuses the fixed scratch array that the first one left behind), and the FP64 oracle's
Delta (Eq. 5), theta (Eq. 4) and F (Eq. 1 at g = 1) within the same tolerances.

This file is collected last so that a run stopping at the first failure has run every other test."""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from gpu_common import assert_matrix_close, theta_tol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available()
    import paper_1210_8018_gb300 as lgf
    f = lgf._lib.lgf_delta_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p]
    return torch, lgf, f


@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (6, 4, 8, 10), (16, 12, 10, 9)])
def test_matches_lgf_delta_twice(env, dims):
    torch, lgf, f = env
    U = synth.config(dims, 61, 0.6)
    with lgf.Lattice(dims) as lat:
        D_ref = np.empty(U.shape[1:], dtype=np.complex128)
        th_ref, F_ref = lat.delta(U, D_ref)
    D_orc = oracle.delta(U)
    th_orc, F_orc = oracle.theta(D_orc), oracle.functional(U)
    Ud = torch.from_numpy(U).to("cuda")
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    for call in range(2):
        D = torch.zeros(U.shape[1:], dtype=torch.complex128, device="cuda")
        tf = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
        st = f(Ud.data_ptr(), *dims, D.data_ptr(), tf.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
        assert st == lgf.LGF_OK, lgf._lib.lgf_last_error(None)
        torch.cuda.synchronize()
        th, F = tf.cpu().numpy()
        Dn = D.cpu().numpy()
        assert_matrix_close(Dn, D_ref)
        assert abs(th - th_ref) <= theta_tol(th_ref), (call, th, th_ref)
        assert abs(F - F_ref) <= 1e-12 * abs(F_ref), (call, F, F_ref)
        assert_matrix_close(Dn, D_orc)
        assert abs(th - th_orc) <= theta_tol(th_orc), (call, th, th_orc)
        assert abs(F - F_orc) <= 1e-12 * abs(F_orc), (call, F, F_orc)


def test_rejects_oversize_and_host_pointers(env):
    torch, lgf, f = env
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    st = f(buf.data_ptr(), 128, 128, 64, 32, None, buf.data_ptr(), None)  # 2^25 sites > 2^24
    assert st == lgf.LGF_EINVAL
    assert b"16777216" in lgf._lib.lgf_last_error(None)
    host = np.zeros(16, dtype=np.float64)
    st = f(host.ctypes.data, 2, 2, 2, 2, None, buf.data_ptr(), None)
    assert st == lgf.LGF_EINVAL
    U = torch.zeros((4, 2, 2, 2, 2, 3, 3), dtype=torch.complex128, device="cuda")
    st = f(U.data_ptr(), 2, 2, 2, 2, None, buf.data_ptr() + 4, None)  # theta_F not 8-byte aligned
    assert st == lgf.LGF_EINVAL and b"aligned" in lgf._lib.lgf_last_error(None)
