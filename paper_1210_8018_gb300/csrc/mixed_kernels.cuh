// mixed_kernels.cuh -- kernels of the mixed-precision schedule: float links, FFTs and updates with the
// accumulated gauge transformation G(x) = g_k(x) ... g_1(x) kept beside them, periodic reprojection of
// the float links and of G onto SU(3) in double precision, and the handover that rebuilds double
// links as G(x) U0_mu(x) G^+(x + mu) from the saved input U0, so that the double-precision stage
// starts from links exactly gauge-equivalent to the input.
#pragma once
#include "site_kernels.cuh"

namespace lgf {

// Float update (as k_update) that also accumulates Gacc(x) <- g(x) Gacc(x).
template <int NT>
__global__ void __launch_bounds__(NT) k_update_accumulate(float *__restrict__ U, const float *__restrict__ G,
                                                         float *__restrict__ Gacc, Lattice L, const Ctrl *ctrl,
                                                         int tkid) {
  if (!ctrl->active) return;
  count_run(ctrl, tkid);
  const int64_t V = L.V;
  const int64_t s = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (s >= V) return;
  int c[4];
  site_coords(L, s, c);
  m3<float> gx, t, a;
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    gx.e[e] = ldg(G, (int64_t)e * V + s);
    a.e[e] = ld(Gacc, (int64_t)e * V + s);
  }
  mul(gx, a, t);
#pragma unroll
  for (int e = 0; e < 9; ++e) st(Gacc, (int64_t)e * V + s, t.e[e]);
#pragma unroll 1
  for (int mu = 0; mu < 4; ++mu) {
    const int64_t sf = site_fwd(L, s, mu, c[mu]);
    float *plane = U + (int64_t)mu * 9 * V * 2;
    m3<float> u, gy;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      u.e[e] = ld(plane, (int64_t)e * V + s);
      gy.e[e] = ldg(G, (int64_t)e * V + sf);
    }
    mul_rows01(gx, u, t);
    mul_adj_rows01(t, gy, u);
    complete_row2(u);
#pragma unroll
    for (int e = 0; e < 9; ++e) st(plane, (int64_t)e * V + s, u.e[e]);
  }
}

// Reproject 5 float matrices per site (4 links and Gacc) onto SU(3) in double precision.
template <int NT>
__global__ void __launch_bounds__(NT) k_reunitarize_fp64(float *__restrict__ U, float *__restrict__ Gacc, int64_t V,
                                                        const Ctrl *ctrl, int tkid) {
  if (!ctrl->active) return;
  count_run(ctrl, tkid);
  const int64_t idx = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (idx >= 5 * V) return;
  const int64_t which = idx / V, s = idx - which * V;
  float *base = which < 4 ? U + which * 9 * V * 2 : Gacc;
  m3<double> m;
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    const cx<float> v = ld(base, (int64_t)e * V + s);
    m.e[e] = {(double)v.r, (double)v.i};
  }
  reunitarize(m);
#pragma unroll
  for (int e = 0; e < 9; ++e) st(base, (int64_t)e * V + s, mkc((float)m.e[e].r, (float)m.e[e].i));
}

// G64 = SU(3)-projection (in double) of the float accumulation.
template <int NT>
__global__ void __launch_bounds__(NT) k_gacc_to_double(const float *__restrict__ Gacc, double *__restrict__ G64,
                                                      int64_t V) {
  const int64_t s = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (s >= V) return;
  m3<double> m;
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    const cx<float> v = ldg(Gacc, (int64_t)e * V + s);
    m.e[e] = {(double)v.r, (double)v.i};
  }
  reunitarize(m);
#pragma unroll
  for (int e = 0; e < 9; ++e) st(G64, (int64_t)e * V + s, m.e[e]);
}

// Udst_mu(x) = G(x) Usrc_mu(x) G^+(x + mu), double precision.
template <int NT>
__global__ void __launch_bounds__(NT) k_transform_from(const double *__restrict__ Usrc, double *__restrict__ Udst,
                                                      const double *__restrict__ G, Lattice L) {
  const int64_t V = L.V;
  const int64_t s = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (s >= V) return;
  int c[4];
  site_coords(L, s, c);
  m3<double> gx;
#pragma unroll
  for (int e = 0; e < 9; ++e) gx.e[e] = ldg(G, (int64_t)e * V + s);
#pragma unroll 1
  for (int mu = 0; mu < 4; ++mu) {
    const int64_t sf = site_fwd(L, s, mu, c[mu]);
    const int64_t off = (int64_t)mu * 9 * V;
    m3<double> u, gy, t;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      u.e[e] = ldg(Usrc, off + (int64_t)e * V + s);
      gy.e[e] = ldg(G, (int64_t)e * V + sf);
    }
    mul(gx, u, t);
    mul_adj(t, gy, u);
#pragma unroll
    for (int e = 0; e < 9; ++e) st(Udst, off + (int64_t)e * V + s, u.e[e]);
  }
}

__global__ void k_set_identity(float *__restrict__ Gacc, int64_t V) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
#pragma unroll
  for (int e = 0; e < 9; ++e) st(Gacc, (int64_t)e * V + s, mkc((e % 4 == 0) ? 1.0f : 0.0f, 0.0f));
}

}  // namespace lgf
