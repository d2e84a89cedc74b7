// mixed_kernels.cuh -- kernels of the mixed-precision schedule: float links, FFTs and updates with the
// accumulated gauge transformation G(x) = g_k(x) ... g_1(x) kept beside them, periodic reprojection of
// the float links and of G onto SU(3), and the handover that rebuilds double
// links as G(x) U0_mu(x) G^+(x + mu) from the saved input U0, so that the double-precision stage
// starts from links exactly gauge-equivalent to the input.
#pragma once
#include "site_kernels.cuh"

namespace lgf {

// g(x) = SU(3)-projection of [1 + (alpha/2) Delta-tilde(x)] from the packed float fields.
__device__ __forceinline__ void gauge_from_packed(const float *P, int64_t V, int64_t s, float half_alpha, m3<float> &g) {
  unpack_scaled(P, V, s, half_alpha, g);
  g.e[0].r += 1.0f;
  g.e[4].r += 1.0f;
  g.e[8].r += 1.0f;
  reunitarize(g);
}

// Float-stage update with g rebuilt in registers: forms g(x) and the four g(x + mu) from the packed
// Delta-tilde (no g field in memory), accumulates Gacc(x) <- g(x) Gacc(x) and applies
// U_mu(x) -> g(x) U_mu(x) g^+(x + mu). With REUNIT the new G and the new links are projected onto SU(3)
// before they are stored (the periodic reunitarisation of the float stage). The projection is done in
// float: it only has to remove the drift from unitarity that float rounding accumulates between
// projections, and the handover rebuilds double links from the saved input and a G projected in double.
template <int NT, bool REUNIT>
__global__ void __launch_bounds__(NT) k_update_fused_f32(float *__restrict__ U, const float *__restrict__ P,
                                                        float *__restrict__ Gacc, float half_alpha, Lattice L,
                                                        const Ctrl *ctrl, int tkid) {
  const int64_t V = L.V;
  {
    const int cfg = blockIdx.z;
    U += (int64_t)cfg * 4 * link_plane_stride<float>(V);
    P += (int64_t)cfg * 4 * V * 2;
    Gacc += (int64_t)cfg * 6 * V * 2;
    ctrl += cfg;
  }
  if (!stage_active<float>(ctrl)) return;
  count_run(ctrl, tkid);
  const int64_t s = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (s >= V) return;
  int c[4];
  site_coords(L, s, c);
  m3<float> gx, t, a;
  gauge_from_packed(P, V, s, half_alpha, gx);
  // G(x) <- g(x) G(x), stored as rows 0 and 1 (like the float links)
#pragma unroll
  for (int e = 0; e < 6; ++e) a.e[e] = ld(Gacc, (int64_t)e * V + s);
  complete_row2(a);
  mul_rows01(gx, a, t);
  if constexpr (REUNIT) reunitarize(t);
#pragma unroll
  for (int e = 0; e < 6; ++e) st(Gacc, (int64_t)e * V + s, t.e[e]);
#pragma unroll 1
  for (int mu = 0; mu < 4; ++mu) {
    const int64_t sf = site_fwd(L, s, mu, c[mu]);
    float *plane = U + (int64_t)mu * link_plane_stride<float>(V);
    m3<float> u, gy;
    load_link(plane, V, s, u);
    gauge_from_packed(P, V, sf, half_alpha, gy);
    mul_rows01(gx, u, t);
    mul_adj_rows01(t, gy, u);
    if constexpr (REUNIT) reunitarize(u);
    store_link(plane, V, s, u);
  }
}

// Float links (rows 0 and 1, 6 planes per direction) from the double link planes (9 per direction),
// rounded to nearest.
__global__ void k_narrow_link_planes(const double *__restrict__ U64, float *__restrict__ U32, int64_t V) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 4 * V) return;
  const int64_t mu = idx / V, s = idx - mu * V;
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    const cx<double> v = ldg(U64, (mu * 9 + e) * V + s);
    st(U32, (mu * 6 + e) * V + s, mkc(narrow_bits(v.r), narrow_bits(v.i)));
  }
}

// G64 = SU(3)-projection (in double) of the float accumulation.
template <int NT>
__global__ void __launch_bounds__(NT) k_gacc_to_double(const float *__restrict__ Gacc, double *__restrict__ G64,
                                                      int64_t V) {
  const int64_t s = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (s >= V) return;
  m3<double> m;
  // rows 0 and 1 of G; the projection rebuilds row 2
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    const cx<float> v = ldg(Gacc, (int64_t)e * V + s);
    m.e[e] = {widen_bits(v.r), widen_bits(v.i)};
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
    mul_rows01(gx, u, t);
    mul_adj_rows01(t, gy, u);
    complete_row2(u);
#pragma unroll
    for (int e = 0; e < 9; ++e) st(Udst, off + (int64_t)e * V + s, u.e[e]);
  }
}

__global__ void k_set_identity(float *__restrict__ Gacc, int64_t V) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
#pragma unroll
  for (int e = 0; e < 6; ++e) st(Gacc, (int64_t)e * V + s, mkc((e % 4 == 0) ? 1.0f : 0.0f, 0.0f));  // rows 0-1
}

}  // namespace lgf
