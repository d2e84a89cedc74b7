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

// SU(3) projection of a float matrix (rows 0-1 given) in double precision; float <-> double by integer
// operations (the conversion instructions would share the FP64 pipe with the projection).
__device__ __forceinline__ void reunitarize_fp64(m3<float> &u) {
  m3<double> d;
#pragma unroll
  for (int e = 0; e < 6; ++e) d.e[e] = {widen_bits(u.e[e].r), widen_bits(u.e[e].i)};
  reunitarize(d);
#pragma unroll
  for (int e = 0; e < 6; ++e) u.e[e] = {narrow_bits(d.e[e].r), narrow_bits(d.e[e].i)};
}

// Float-stage update with g rebuilt in registers: forms g(x) and the four g(x + mu) from the packed
// Delta-tilde (no g field in memory), accumulates Gacc(x) <- g(x) Gacc(x) and applies
// U_mu(x) -> g(x) U_mu(x) g^+(x + mu). With REUNIT the new G and the new links are projected onto SU(3)
// before they are stored (the periodic reunitarisation of the float stage): REUNIT 1 projects in float,
// which only has to remove the drift from unitarity that float rounding accumulates between projections
// (the handover rebuilds double links from the saved input and a G projected in double); REUNIT 2
// projects in double precision.
template <int NT, int REUNIT>
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
  if constexpr (REUNIT == 1) reunitarize(t);
  if constexpr (REUNIT == 2) reunitarize_fp64(t);
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
    if constexpr (REUNIT == 1) reunitarize(u);
    if constexpr (REUNIT == 2) reunitarize_fp64(u);
    store_link(plane, V, s, u);
  }
}

// The same update walking along t: thread (x, y, z) takes the TCH consecutive t-slices of chunk blockIdx.y
// one after another. The g(x + t) it forms for the links U_t is the g(x) of its next slice, kept in
// registers: every t-neighbour's Delta-tilde is read and projected once instead of twice (in site order the
// second read comes a whole 3D slice later, after about 140 MB of other traffic at 64^4, and misses the L2).
// Same arithmetic per site as k_update_fused_f32 (measured at 64^4: 1.47 -> 1.37 ms). Needs Nt % TCH == 0.
template <int NT, int REUNIT, int TCH>
__global__ void __launch_bounds__(NT) k_update_fused_f32_tw(float *__restrict__ U, const float *__restrict__ P,
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
  const int64_t nxyz = L.stride[3];
  const int64_t q = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (q >= nxyz) return;
  const int t0 = blockIdx.y * TCH;
  int c[4];
  site_coords(L, q + (int64_t)t0 * nxyz, c);
  // U_mu(x) <- g(x) U_mu(x) g(y)^dagger, projected like the float links
  auto link_update = [&](float *plane, int64_t s, const m3<float> &gx, const m3<float> &gy) {
    m3<float> u, tm;
    load_link(plane, V, s, u);
    mul_rows01(gx, u, tm);
    mul_adj_rows01(tm, gy, u);
    if constexpr (REUNIT == 1) reunitarize(u);
    if constexpr (REUNIT == 2) reunitarize_fp64(u);
    store_link(plane, V, s, u);
  };
  m3<float> gx;
  gauge_from_packed(P, V, q + (int64_t)t0 * nxyz, half_alpha, gx);
#pragma unroll 1
  for (int k = 0; k < TCH; ++k) {
    const int t = t0 + k;
    const int64_t s = q + (int64_t)t * nxyz;
    {
      m3<float> a, tm;
      // G(x) <- g(x) G(x), stored as rows 0 and 1 (like the float links)
#pragma unroll
      for (int e = 0; e < 6; ++e) a.e[e] = ld(Gacc, (int64_t)e * V + s);
      complete_row2(a);
      mul_rows01(gx, a, tm);
      if constexpr (REUNIT == 1) reunitarize(tm);
      if constexpr (REUNIT == 2) reunitarize_fp64(tm);
#pragma unroll
      for (int e = 0; e < 6; ++e) st(Gacc, (int64_t)e * V + s, tm.e[e]);
    }
#pragma unroll 1
    for (int mu = 0; mu < 3; ++mu) {
      m3<float> gy;
      gauge_from_packed(P, V, site_fwd(L, s, mu, c[mu]), half_alpha, gy);
      link_update(U + (int64_t)mu * link_plane_stride<float>(V), s, gx, gy);
    }
    m3<float> gt;  // g(x + t), the g(x) of the next slice
    gauge_from_packed(P, V, q + (int64_t)(t + 1 == L.n[3] ? 0 : t + 1) * nxyz, half_alpha, gt);
    link_update(U + (int64_t)3 * link_plane_stride<float>(V), s, gx, gt);
    gx = gt;
  }
}

// Float links (rows 0 and 1, 6 planes per direction) from the double link planes (9 per direction),
// rounded to nearest.
__global__ void k_narrow_link_planes(const double *__restrict__ U64, float *__restrict__ U32, int64_t V, int64_t idx0,
                                     int64_t n) {
  const int64_t idx = idx0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= idx0 + n || idx >= 4 * V) return;
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

// Udst_mu(x) = G(x) Usrc_mu(x) G^+(x + mu), double precision; with U32, rows 0-1 of the result also
// rounded to float into the float link planes (the base of the residual stage).
template <int NT>
__global__ void __launch_bounds__(NT) k_transform_from(const double *__restrict__ Usrc, double *__restrict__ Udst,
                                                      const double *__restrict__ G, Lattice L,
                                                      float *__restrict__ U32) {
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
    if (U32) {
#pragma unroll
      for (int e = 0; e < 6; ++e)
        st(U32, (int64_t)(mu * 6 + e) * V + s, mkc(narrow_bits(u.e[e].r), narrow_bits(u.e[e].i)));
    }
  }
}

// Q61 arithmetic (to_q61, mul_q61, cq_mac, from_q61, ...): q61.cuh.

// The link mu of site s in FP64: Udst = G(x) Usrc G^+(x + mu), rows 0-1 by products, row 2 = conj(row0 x row1).
__device__ __forceinline__ void transform_link_fp64(const double *__restrict__ Usrc, double *__restrict__ Udst,
                                                    const double *__restrict__ G, int64_t V, int64_t s, int64_t sf,
                                                    int64_t off, float *__restrict__ U32, int mu) {
  m3<double> gx, u, gy, t;
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    gx.e[e] = e < 6 ? ldg(G, (int64_t)e * V + s) : cx<double>{0.0, 0.0};  // rows 0-1 are used
    u.e[e] = ldg(Usrc, off + (int64_t)e * V + s);
    gy.e[e] = ldg(G, (int64_t)e * V + sf);
  }
  mul_rows01(gx, u, t);
  mul_adj_rows01(t, gy, u);
  complete_row2(u);
#pragma unroll
  for (int e = 0; e < 9; ++e) st(Udst, off + (int64_t)e * V + s, u.e[e]);
  if (U32) {
#pragma unroll
    for (int e = 0; e < 6; ++e) st(U32, (int64_t)(mu * 6 + e) * V + s, mkc(narrow_bits(u.e[e].r), narrow_bits(u.e[e].i)));
  }
}

// The four links of a site split between the two forms: the first fp64_even (in even warps) or fp64_odd
// (in odd warps) directions in FP64, the others in Q61. The FP64 pipe and the integer pipes then work at
// the same time on different warps; both forms are exact to FP64 rounding. fp64_even = fp64_odd = 0 is
// the fixed-point form alone.
template <int NT>
__global__ void __launch_bounds__(NT, 2) k_transform_from_q(const double *__restrict__ Usrc, double *__restrict__ Udst,
                                                        const double *__restrict__ G, Lattice L,
                                                        float *__restrict__ U32, int fp64_even, int fp64_odd) {
  const int64_t V = L.V;
  const int64_t s = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (s >= V) return;
  int c[4];
  site_coords(L, s, c);
  const int nf = ((threadIdx.x >> 5) & 1) ? fp64_odd : fp64_even;  // uniform within a warp
  cq gx[6];  // rows 0-1 of G(x): the rows of the result that are formed (row 2 follows from them)
#pragma unroll
  for (int e = 0; e < 6; ++e) gx[e] = to_cq(ldg(G, (int64_t)e * V + s));
#pragma unroll 1
  for (int mu = 0; mu < 4; ++mu) {
    const int64_t sf = site_fwd(L, s, mu, c[mu]);
    const int64_t off = (int64_t)mu * 9 * V;
    if (mu < nf) {
      transform_link_fp64(Usrc, Udst, G, V, s, sf, off, U32, mu);
      continue;
    }
    cq t[6], o[9];
    // rows 0-1 of G(x) U, one column of U at a time
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const cq u0 = to_cq(ldg(Usrc, off + (int64_t)j * V + s));
      const cq u1 = to_cq(ldg(Usrc, off + (int64_t)(3 + j) * V + s));
      const cq u2 = to_cq(ldg(Usrc, off + (int64_t)(6 + j) * V + s));
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        cq a = {0, 0};
        cq_mac(a, gx[3 * i], u0);
        cq_mac(a, gx[3 * i + 1], u1);
        cq_mac(a, gx[3 * i + 2], u2);
        t[3 * i + j] = a;
      }
    }
    // rows 0-1 of (G U) G^+(x + mu), one row of G(x + mu) at a time
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const cq g0 = to_cq(ldg(G, (int64_t)(3 * j) * V + sf));
      const cq g1 = to_cq(ldg(G, (int64_t)(3 * j + 1) * V + sf));
      const cq g2 = to_cq(ldg(G, (int64_t)(3 * j + 2) * V + sf));
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        cq a = {0, 0};
        cq_mac_cj(a, t[3 * i], g0);
        cq_mac_cj(a, t[3 * i + 1], g1);
        cq_mac_cj(a, t[3 * i + 2], g2);
        o[3 * i + j] = a;
      }
    }
    o[6] = cq_cross_cj(o[1], o[5], o[2], o[4]);
    o[7] = cq_cross_cj(o[2], o[3], o[0], o[5]);
    o[8] = cq_cross_cj(o[0], o[4], o[1], o[3]);
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      const cx<double> v = {from_q61(o[e].r), from_q61(o[e].i)};
      st(Udst, off + (int64_t)e * V + s, v);
      if (U32 && e < 6) st(U32, (int64_t)(mu * 6 + e) * V + s, mkc(narrow_bits(v.r), narrow_bits(v.i)));
    }
  }
}

__global__ void k_set_identity(float *__restrict__ Gacc, int64_t V) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
#pragma unroll
  for (int e = 0; e < 6; ++e) st(Gacc, (int64_t)e * V + s, mkc((e % 4 == 0) ? 1.0f : 0.0f, 0.0f));  // rows 0-1
}

// ---------------------------------------------------------------------------------------------
// Residual stage of the mixed schedule (after the handover). The links are U = U_h + R: U_h are the
// handover links (double, fixed for the stage) and R, a float residual starting at zero, takes every
// change. Delta is linear in the links, so Delta(U) = Delta(U_h) + Delta(R) with Delta(U_h) computed
// once in double. The update needs U only to float accuracy (it multiplies the small a and b), and
// reads it as B + R with B = U_h rounded to float (rows 0-1, the float link planes). Every float
// quantity of the stage (a = g - 1, R, K with H = 1 + K the transformation gathered in the stage) is of
// the size of the remaining gauge transformation, so its rounding is relative to that size and not to
// the O(1) links: with changes of order 1e-4 the links are tracked to about 1e-11 and Delta to about
// 1e-10, against entries of 3e-8 at theta = 1e-15. The stage ends with H projected onto SU(3) in double
// and U_h -> H U_h H^+(x + mu) by the double update (k_update, whose small-step form is exact to FP64
// rounding for H close to 1), so the result stays exactly gauge-equivalent to the input; theta is then
// recomputed in double.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ bool residual_active(const Ctrl *ctrl) {
  return ctrl->active && ctrl->stage == kStageResidual;
}

__device__ __forceinline__ float packed_to_float(df64 v) { return __fadd_rn(v.hi, v.lo); }
__device__ __forceinline__ float packed_to_float(double v) { return narrow_bits(v); }

template <typename T> __device__ __forceinline__ void load9(const T *plane, int64_t V, int64_t s, m3<T> &u) {
#pragma unroll
  for (int e = 0; e < 9; ++e) u.e[e] = ldg(plane, (int64_t)e * V + s);
}

// Delta = Delta(U_h) + Delta(R) (packed, float), theta and F = F(U_h) + sum Re Tr R / (12 V) (a1/a2),
// F(U_h) from the loop control. Ph: packed Delta(U_h) in the double state's FFT type PT. blockIdx.z:
// configuration of a batch group.
// (four resident blocks per SM asked of the compiler: 64 registers instead of 72, 32 warps in flight instead
// of 24; measured at 64^4: 1.26 -> 1.11 ms per launch)
template <int NT, typename PT>
__global__ void __launch_bounds__(NT, 4) k_delta_residual(const float *__restrict__ R, const PT *__restrict__ Ph,
                                                      float *__restrict__ P, double *partials, Ctrl *ctrl, Lattice L,
                                                      int counts_update, int tkid) {
  const int64_t V = L.V;
  {
    const int cfg = blockIdx.z;
    R += (int64_t)cfg * 36 * V * 2;
    Ph += (int64_t)cfg * 4 * V * 2;
    P += (int64_t)cfg * 4 * V * 2;
    partials += (int64_t)cfg * 2 * gridDim.x;
    ctrl += cfg;
  }
  if (!residual_active(ctrl)) return;
  count_run(ctrl, tkid);
  double th = 0.0, f = 0.0;
#pragma unroll 1
  for (int k = 0; k < kSitesPerThread; ++k) {
    const int64_t s = ((int64_t)blockIdx.x * kSitesPerThread + k) * NT + threadIdx.x;
    if (s >= V) break;
    int c[4];
    site_coords(L, s, c);
    float acc[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) acc[e] = 0.f;
    float fs = 0.f;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      const float *plane = R + (int64_t)mu * 18 * V;
      m3<float> u;
      load9(plane, V, site_back(L, s, mu, c[mu]), u);  // R_mu(x - mu)
      accumulate_link(u, 1.f, acc);
      load9(plane, V, s, u);  // - R_mu(x)
      accumulate_link(u, -1.f, acc);
      fs += u.e[0].r + u.e[4].r + u.e[8].r;
    }
    const float m = (acc[6] + acc[7] + acc[8]) / 3.f;
    float d[8] = {acc[0], acc[1], acc[2], acc[3], acc[4], acc[5], 2.f * (acc[6] - m), 2.f * (acc[7] - m)};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const cx<PT> h = ldg(Ph, (int64_t)q * V + s);
      d[2 * q] += packed_to_float(h.r);
      d[2 * q + 1] += packed_to_float(h.i);
    }
    const float a2 = -(d[6] + d[7]);
    const float ts = d[6] * d[6] + d[7] * d[7] + a2 * a2 +
                     2.f * (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + d[3] * d[3] + d[4] * d[4] + d[5] * d[5]);
    th += widen_bits(ts);
    f += widen_bits(fs);
#pragma unroll
    for (int q = 0; q < 4; ++q) st(P, (int64_t)q * V + s, mkc(d[2 * q], d[2 * q + 1]));
  }
  reduce_and_finalize<NT>(th, f, partials, ctrl, V, counts_update, ctrl->f_base);
}

// The same residual Delta walking along t (as k_delta_f32_tw): the combinations of R_t(x) accumulated
// for one slice are those of the backward link R_t(x - t) of the next, kept in registers, so seven
// residual links are read per site instead of eight. Same sums in the same order (Delta the same bits).
// Measured at 64^4: 1.10 -> 1.02 ms. Needs Nt % TCH == 0.
template <int NT, typename PT, int TCH>
__global__ void __launch_bounds__(NT, 4) k_delta_residual_tw(const float *__restrict__ R, const PT *__restrict__ Ph,
                                                         float *__restrict__ P, double *partials, Ctrl *ctrl,
                                                         Lattice L, int counts_update, int tkid) {
  const int64_t V = L.V;
  const unsigned nblk = gridDim.x * gridDim.y;
  {
    const int cfg = blockIdx.z;
    R += (int64_t)cfg * 36 * V * 2;
    Ph += (int64_t)cfg * 4 * V * 2;
    P += (int64_t)cfg * 4 * V * 2;
    partials += (int64_t)cfg * 2 * nblk;
    ctrl += cfg;
  }
  if (!residual_active(ctrl)) return;
  count_run(ctrl, tkid);
  const int64_t nxyz = L.stride[3];
  const int64_t q = (int64_t)blockIdx.x * NT + threadIdx.x;
  double th = 0.0, f = 0.0;
  if (q < nxyz) {
    const int t0 = blockIdx.y * TCH;
    int c[4];
    site_coords(L, q + (int64_t)t0 * nxyz, c);
    const float *plane_t = R + (int64_t)3 * 18 * V;
    float tb[9];  // combinations of R_t(x - t): the previous slice's R_t(x)
    {
      m3<float> u;
      load9(plane_t, V, site_back(L, q + (int64_t)t0 * nxyz, 3, t0), u);
#pragma unroll
      for (int e = 0; e < 9; ++e) tb[e] = 0.f;
      accumulate_link(u, 1.f, tb);
    }
#pragma unroll 1
    for (int k = 0; k < TCH; ++k) {
      const int64_t s = q + (int64_t)(t0 + k) * nxyz;
      float acc[9];
#pragma unroll
      for (int e = 0; e < 9; ++e) acc[e] = 0.f;
      float fs = 0.f;
#pragma unroll
      for (int mu = 0; mu < 3; ++mu) {
        const float *plane = R + (int64_t)mu * 18 * V;
        m3<float> u;
        load9(plane, V, site_back(L, s, mu, c[mu]), u);  // R_mu(x - mu)
        accumulate_link(u, 1.f, acc);
        load9(plane, V, s, u);  // - R_mu(x)
        accumulate_link(u, -1.f, acc);
        fs += u.e[0].r + u.e[4].r + u.e[8].r;
      }
      {
        m3<float> u;
        load9(plane_t, V, s, u);
#pragma unroll
        for (int e = 0; e < 9; ++e) acc[e] = fmaf(1.f, tb[e], acc[e]);  // + R_t(x - t)
        accumulate_link(u, -1.f, acc);                                   // - R_t(x)
        fs += u.e[0].r + u.e[4].r + u.e[8].r;
#pragma unroll
        for (int e = 0; e < 9; ++e) tb[e] = 0.f;
        accumulate_link(u, 1.f, tb);
      }
      const float m = (acc[6] + acc[7] + acc[8]) / 3.f;
      float d[8] = {acc[0], acc[1], acc[2], acc[3], acc[4], acc[5], 2.f * (acc[6] - m), 2.f * (acc[7] - m)};
#pragma unroll
      for (int qq = 0; qq < 4; ++qq) {
        const cx<PT> h = ldg(Ph, (int64_t)qq * V + s);
        d[2 * qq] += packed_to_float(h.r);
        d[2 * qq + 1] += packed_to_float(h.i);
      }
      const float a2 = -(d[6] + d[7]);
      const float ts = d[6] * d[6] + d[7] * d[7] + a2 * a2 +
                       2.f * (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + d[3] * d[3] + d[4] * d[4] + d[5] * d[5]);
      th += widen_bits(ts);
      f += widen_bits(fs);
#pragma unroll
      for (int qq = 0; qq < 4; ++qq) st(P, (int64_t)qq * V + s, mkc(d[2 * qq], d[2 * qq + 1]));
    }
  }
  reduce_and_finalize_at<NT>(th, f, partials, ctrl, V, counts_update, ctrl->f_base,
                             blockIdx.x + gridDim.x * blockIdx.y, nblk);
}

// Loop control of one configuration entering the residual stage (after its double Delta, theta and F):
// F of the base, the stage and its threshold, active.
__global__ void k_enter_residual(Ctrl *ctrl, double threshold) {
  ctrl->f_base = ctrl->F;
  ctrl->stage = kStageResidual;
  ctrl->threshold = threshold;
  ctrl->active = 1;
}

__global__ void k_set_active(Ctrl *ctrl, int active) { ctrl->active = active; }

// a = g - 1 with g the SU(3) projection of 1 + X, in float: the small-step form when every |X| < 2^-8,
// else Gram-Schmidt of 1 + X minus the identity (large steps, where float rounding of a is harmless).
__device__ __forceinline__ void residual_step(const m3<float> &X, m3<float> &a) {
  float mx = 0.f;
#pragma unroll
  for (int e = 0; e < 9; ++e) mx = fmaxf(mx, fmaxf(fabsf(X.e[e].r), fabsf(X.e[e].i)));
  if (mx < 0x1p-8f) {
    small_step_projection(X, a);
    return;
  }
  a = X;
  a.e[0].r += 1.f;
  a.e[4].r += 1.f;
  a.e[8].r += 1.f;
  reunitarize(a);
  a.e[0].r -= 1.f;
  a.e[4].r -= 1.f;
  a.e[8].r -= 1.f;
}

// a6 + a7 on the residual: a(x) and b = g(x + mu) - 1 from the packed Delta-tilde (float), K <- a + K + a K
// (H <- g H), and R_mu(x) <- R_mu(x) + a U + (U + a U) b^+ with U = B + R (U -> g U g^+(x + mu)).
// B: float link planes (rows 0-1; row 2 completed on load).
template <int NT>
__global__ void __launch_bounds__(NT) k_update_residual(const float *__restrict__ B, float *__restrict__ R,
                                                       float *__restrict__ K, const float *__restrict__ P,
                                                       float half_alpha, Lattice L, const Ctrl *ctrl, int tkid) {
  const int64_t V = L.V;
  {
    const int cfg = blockIdx.z;
    B += (int64_t)cfg * 4 * link_plane_stride<float>(V);
    R += (int64_t)cfg * 36 * V * 2;
    K += (int64_t)cfg * 9 * V * 2;
    P += (int64_t)cfg * 4 * V * 2;
    ctrl += cfg;
  }
  if (!residual_active(ctrl)) return;
  count_run(ctrl, tkid);
  const int64_t s = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (s >= V) return;
  m3<float> X, a, t;
  unpack_scaled(P, V, s, half_alpha, X);
  residual_step(X, a);
  {
    m3<float> k;
    load9(K, V, s, k);
    mul(a, k, t);
#pragma unroll
    for (int e = 0; e < 9; ++e) st(K, (int64_t)e * V + s, (a.e[e] + k.e[e]) + t.e[e]);
  }
#pragma unroll 1
  for (int mu = 0; mu < 4; ++mu) {
    m3<float> b, u, r, w;
    const int cmu = (int)(((unsigned)s / (unsigned)L.stride[mu]) % (unsigned)L.n[mu]);
    unpack_scaled(P, V, site_fwd(L, s, mu, cmu), half_alpha, X);
    residual_step(X, b);
    float *rp = R + (int64_t)mu * 18 * V;
    load9(rp, V, s, r);
    load_link(B + (int64_t)mu * link_plane_stride<float>(V), V, s, u);
#pragma unroll
    for (int e = 0; e < 9; ++e) u.e[e] = u.e[e] + r.e[e];
    mul(a, u, t);  // a U
#pragma unroll
    for (int e = 0; e < 9; ++e) w.e[e] = u.e[e] + t.e[e];  // g U
    mul_adj(w, b, u);                                      // (g U) b^+
#pragma unroll
    for (int e = 0; e < 9; ++e) st(rp, (int64_t)e * V + s, r.e[e] + (t.e[e] + u.e[e]));
  }
}

// The same residual update walking along t (as k_update_fused_f32_tw): thread (x, y, z) takes the TCH
// t-slices of chunk blockIdx.y, and the b formed for its links U_t is the a of its next slice, so each
// t-neighbour's Delta-tilde is read and projected once. Same arithmetic per site (measured at 64^4: 2.96 ->
// 2.82 ms). Needs Nt % TCH == 0.
template <int NT, int TCH>
__global__ void __launch_bounds__(NT, 2) k_update_residual_tw(const float *__restrict__ B, float *__restrict__ R,
                                                          float *__restrict__ K, const float *__restrict__ P,
                                                          float half_alpha, Lattice L, const Ctrl *ctrl, int tkid) {
  const int64_t V = L.V;
  {
    const int cfg = blockIdx.z;
    B += (int64_t)cfg * 4 * link_plane_stride<float>(V);
    R += (int64_t)cfg * 36 * V * 2;
    K += (int64_t)cfg * 9 * V * 2;
    P += (int64_t)cfg * 4 * V * 2;
    ctrl += cfg;
  }
  if (!residual_active(ctrl)) return;
  count_run(ctrl, tkid);
  const int64_t nxyz = L.stride[3];
  const int64_t q = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (q >= nxyz) return;
  const int t0 = blockIdx.y * TCH;
  int c[4];
  site_coords(L, q + (int64_t)t0 * nxyz, c);
  // R_mu(x) <- R_mu(x) + a U + (U + a U) b^+ with U = B + R
  auto link_update = [&](int mu, int64_t s, const m3<float> &a, const m3<float> &b) {
    m3<float> u, r, w, t;
    float *rp = R + (int64_t)mu * 18 * V;
    load9(rp, V, s, r);
    load_link(B + (int64_t)mu * link_plane_stride<float>(V), V, s, u);
#pragma unroll
    for (int e = 0; e < 9; ++e) u.e[e] = u.e[e] + r.e[e];
    mul(a, u, t);  // a U
#pragma unroll
    for (int e = 0; e < 9; ++e) w.e[e] = u.e[e] + t.e[e];  // g U
    mul_adj(w, b, u);                                      // (g U) b^+
#pragma unroll
    for (int e = 0; e < 9; ++e) st(rp, (int64_t)e * V + s, r.e[e] + (t.e[e] + u.e[e]));
  };
  m3<float> a;
  {
    m3<float> X;
    unpack_scaled(P, V, q + (int64_t)t0 * nxyz, half_alpha, X);
    residual_step(X, a);
  }
#pragma unroll 1
  for (int k = 0; k < TCH; ++k) {
    const int t = t0 + k;
    const int64_t s = q + (int64_t)t * nxyz;
    {
      m3<float> kk, tm;
      load9(K, V, s, kk);
      mul(a, kk, tm);
#pragma unroll
      for (int e = 0; e < 9; ++e) st(K, (int64_t)e * V + s, (a.e[e] + kk.e[e]) + tm.e[e]);
    }
#pragma unroll 1
    for (int mu = 0; mu < 3; ++mu) {
      m3<float> X, b;
      unpack_scaled(P, V, site_fwd(L, s, mu, c[mu]), half_alpha, X);
      residual_step(X, b);
      link_update(mu, s, a, b);
    }
    m3<float> bt;  // b of the link U_t: the a of the next slice
    {
      m3<float> X;
      unpack_scaled(P, V, q + (int64_t)(t + 1 == L.n[3] ? 0 : t + 1) * nxyz, half_alpha, X);
      residual_step(X, bt);
    }
    link_update(3, s, a, bt);
    a = bt;
  }
}

// H = proj(1 + K) into G (double) and a = H - 1 in double-float into A: the gauge field with which the
// double update (small-step form) rebuilds U_h -> H U_h H^+(x + mu). K is the transformation gathered in the
// residual stage, of the size of the remaining gauge rotation (about 1e-4): per warp, when every |K_ij| of
// rows 0-1 is below 2^-8, the small-step projection of the double path (a from small quantities in
// double-float, g = 1 + a assembled in FP64, exact to FP64 rounding) replaces Gram-Schmidt in FP64.
template <int NT>
__global__ void __launch_bounds__(NT) k_residual_gauge(const float *__restrict__ K, double *__restrict__ G,
                                                      float *__restrict__ A, int64_t V) {
  const int64_t s = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (s >= V) return;
  {
    m3<df64> X, a;
    int ef = 0;
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      const cx<float> k = ldg(K, (int64_t)e * V + s);
      X.e[e] = {df64{k.r, 0.f}, df64{k.i, 0.f}};
      ef = max(ef, max(fexp_field(k.r), fexp_field(k.i)));
    }
    if (__all_sync(__activemask(), ef <= kSmallXFloatExpField)) {
      small_step_projection(X, a);
#pragma unroll
      for (int e = 0; e < 9; ++e) {
        double re = convert<double>(a.e[e].r);
        if (e == 0 || e == 4 || e == 8) re = 1.0 + re;
        st(G, (int64_t)e * V + s, mkc(re, convert<double>(a.e[e].i)));
        st_a(A, (int64_t)e * V + s, a.e[e]);
      }
      return;
    }
  }
  m3<double> h;
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    const cx<float> k = ldg(K, (int64_t)e * V + s);
    h.e[e] = {widen_bits(k.r), widen_bits(k.i)};
  }
  h.e[0].r += 1.0;
  h.e[4].r += 1.0;
  h.e[8].r += 1.0;
  reunitarize(h);
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    st(G, (int64_t)e * V + s, h.e[e]);
    st_a(A, (int64_t)e * V + s, minus_identity_split(h.e[e], e));
  }
}

}  // namespace lgf
