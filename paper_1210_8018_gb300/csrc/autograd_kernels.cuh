// autograd_kernels.cuh -- the gauge functional as a differentiable function of a Lie-algebra field:
//   F(omega) = F_U[g] with g(x) = exp(i omega(x)), omega(x) = sum_a omega^a(x) T^a, T^a = lambda^a / 2
// (Eq. 1 of the paper evaluated at g = exp(i omega)), and its gradient dF/d omega^a(x), the
// steepest-ascent direction that the Fourier-accelerated method preconditions.
//
// Gradient: g(x) enters F through Re Tr[g(x) K(x)] with the staple
//   K(x) = sum_mu [ U_mu(x) g^+(x+mu) + U_mu^+(x-mu) g^+(x-mu) ].
// With omega = W diag(l) W^+, the derivative of the matrix exponential (Daleckii-Krein) gives
//   dF/d omega^a = -(1/(12 V)) Im Tr[ T^a W (Phi o (W^+ K W)) W^+ ],
//   Phi_jk = exp(i (l_j + l_k)/2) sinc((l_j - l_k)/2)   (the divided difference of exp(i l)),
// which is stable for (near-)degenerate eigenvalues. At omega = 0 it reduces to
// -(i/(24 V)) Tr[T^a Delta(x)] with Delta of Eq. 5.
#pragma once
#include "site_kernels.cuh"

namespace lgf {

// Hermitian matrix H = sum_a w^a lambda^a / 2.
__device__ __forceinline__ void algebra_matrix(const double w[8], m3<double> &H) {
  const double s3 = 0.57735026918962576451;  // 1/sqrt(3)
  H.e[0] = {0.5 * (w[2] + s3 * w[7]), 0};
  H.e[4] = {0.5 * (-w[2] + s3 * w[7]), 0};
  H.e[8] = {-s3 * w[7], 0};
  H.e[1] = {0.5 * w[0], -0.5 * w[1]};
  H.e[3] = {0.5 * w[0], 0.5 * w[1]};
  H.e[2] = {0.5 * w[3], -0.5 * w[4]};
  H.e[6] = {0.5 * w[3], 0.5 * w[4]};
  H.e[5] = {0.5 * w[5], -0.5 * w[6]};
  H.e[7] = {0.5 * w[5], 0.5 * w[6]};
}

// Cyclic Jacobi eigen-decomposition of a Hermitian 3x3 matrix: H = W diag(l) W^+ (W unitary).
// Each rotation first makes H_pq real with a phase on column q, then applies the real Jacobi rotation.
// At most 12 sweeps (quadratic convergence; 4-5 are used in practice).
__device__ __forceinline__ void jacobi_eigh(m3<double> H, m3<double> &W, double l[3]) {
  for (int e = 0; e < 9; ++e) W.e[e] = {(e % 4 == 0) ? 1.0 : 0.0, 0.0};
  const double scale = sqrt(norm2(H.e[0]) + norm2(H.e[4]) + norm2(H.e[8]) +
                            2.0 * (norm2(H.e[1]) + norm2(H.e[2]) + norm2(H.e[5]))) + 1e-300;
  for (int sweep = 0; sweep < 12; ++sweep) {
    const double off = norm2(H.e[1]) + norm2(H.e[2]) + norm2(H.e[5]);
    if (off <= 1e-34 * scale * scale) break;
    for (int pq = 0; pq < 3; ++pq) {
      const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
      const cx<double> h = H.e[3 * p + q];
      const double r = sqrt(norm2(h));
      if (r <= 1e-300) continue;
      // phase: column q times d = conj(h)/r, row q times conj(d) -> H_pq becomes r (real)
      const cx<double> d = {h.r / r, -h.i / r};
      for (int k = 0; k < 3; ++k) {
        H.e[3 * k + q] = H.e[3 * k + q] * d;
        W.e[3 * k + q] = W.e[3 * k + q] * d;
      }
      for (int k = 0; k < 3; ++k) H.e[3 * q + k] = H.e[3 * q + k] * conjg(d);
      // real rotation on (p, q)
      const double app = H.e[3 * p + p].r, aqq = H.e[3 * q + q].r;
      const double tau = (aqq - app) / (2.0 * r);
      const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
      const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
      // columns: H <- H R, W <- W R with R = [[c, s], [-s, c]] on (p, q)
      for (int k = 0; k < 3; ++k) {
        const cx<double> hp = H.e[3 * k + p], hq = H.e[3 * k + q];
        H.e[3 * k + p] = {c * hp.r - s * hq.r, c * hp.i - s * hq.i};
        H.e[3 * k + q] = {s * hp.r + c * hq.r, s * hp.i + c * hq.i};
        const cx<double> wp = W.e[3 * k + p], wq = W.e[3 * k + q];
        W.e[3 * k + p] = {c * wp.r - s * wq.r, c * wp.i - s * wq.i};
        W.e[3 * k + q] = {s * wp.r + c * wq.r, s * wp.i + c * wq.i};
      }
      // rows: H <- R^T H
      for (int k = 0; k < 3; ++k) {
        const cx<double> hp = H.e[3 * p + k], hq = H.e[3 * q + k];
        H.e[3 * p + k] = {c * hp.r - s * hq.r, c * hp.i - s * hq.i};
        H.e[3 * q + k] = {s * hp.r + c * hq.r, s * hp.i + c * hq.i};
      }
      H.e[3 * p + q] = {0, 0};
      H.e[3 * q + p] = {0, 0};
    }
  }
  l[0] = H.e[0].r;
  l[1] = H.e[4].r;
  l[2] = H.e[8].r;
}

// g = W diag(exp(i l)) W^+
__device__ __forceinline__ void expi_from_eig(const m3<double> &W, const double l[3], m3<double> &g) {
  cx<double> ph[3];
  for (int k = 0; k < 3; ++k) {
    double sn, cs;
    sincos(l[k], &sn, &cs);
    ph[k] = {cs, sn};
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      cx<double> acc = {0, 0};
      for (int k = 0; k < 3; ++k) acc = cmac_cj(acc, W.e[3 * i + k] * ph[k], W.e[3 * j + k]);
      g.e[3 * i + j] = acc;
    }
}

// omega (V x 8, site-major) -> g (9 planes), W (9 planes), eigenvalues (3 planes of doubles).
template <int NT>
__global__ void __launch_bounds__(NT) k_expi(const double *__restrict__ omega, double *__restrict__ G,
                                            double *__restrict__ Wp, double *__restrict__ lam, int64_t V) {
  const int64_t s = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (s >= V) return;
  double w[8];
  for (int a = 0; a < 8; ++a) w[a] = omega[s * 8 + a];
  m3<double> H, W, g;
  algebra_matrix(w, H);
  double l[3];
  jacobi_eigh(H, W, l);
  expi_from_eig(W, l, g);
  for (int e = 0; e < 9; ++e) {
    st(G, (int64_t)e * V + s, g.e[e]);
    st(Wp, (int64_t)e * V + s, W.e[e]);
  }
  for (int k = 0; k < 3; ++k) lam[(int64_t)k * V + s] = l[k];
}

// F partials: sum_mu Re Tr[g(x) U_mu(x) g^+(x+mu)] per site, reduced in FP64 (kSitesPerThread sites per
// thread, the grid of k_delta).
template <int NT>
__global__ void __launch_bounds__(NT) k_functional_g(const double *__restrict__ U, const double *__restrict__ G,
                                                    double *partials, Ctrl *ctrl, Lattice L) {
  const int64_t V = L.V;
  double f = 0.0;
  for (int k = 0; k < kSitesPerThread; ++k) {
    const int64_t s = ((int64_t)blockIdx.x * kSitesPerThread + k) * NT + threadIdx.x;
    if (s >= V) break;
    int c[4];
    site_coords(L, s, c);
    m3<double> gx;
    for (int e = 0; e < 9; ++e) gx.e[e] = ldg(G, (int64_t)e * V + s);
    for (int mu = 0; mu < 4; ++mu) {
      const int64_t sf = site_fwd(L, s, mu, c[mu]);
      const double *plane = U + (int64_t)mu * 9 * V * 2;
      m3<double> u, t;
      for (int e = 0; e < 9; ++e) u.e[e] = ldg(plane, (int64_t)e * V + s);
      mul(gx, u, t);
      for (int e = 0; e < 9; ++e) {  // Re Tr[t g'^+] = sum_ij Re(t_ij conj(g'_ij))
        const cx<double> gy = ldg(G, (int64_t)e * V + sf);
        f += t.e[e].r * gy.r + t.e[e].i * gy.i;
      }
    }
  }
  double th = 0.0;
  reduce_and_finalize<NT>(th, f, partials, ctrl, V, 0);
}

__device__ __forceinline__ double sinc_half(double x) {  // sin(x)/x
  const double ax = fabs(x);
  if (ax < 1e-4) {
    const double x2 = x * x;
    return 1.0 - x2 / 6.0 + x2 * x2 / 120.0;
  }
  return sin(x) / x;
}

// dF/d omega^a(x), a = 0..7, written site-major (V x 8), scaled by `scale` (the incoming gradient).
template <int NT>
__global__ void __launch_bounds__(NT) k_functional_grad(const double *__restrict__ U, const double *__restrict__ G,
                                                       const double *__restrict__ Wp, const double *__restrict__ lam,
                                                       double *__restrict__ grad, Lattice L, double scale) {
  const int64_t V = L.V;
  const int64_t s = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (s >= V) return;
  int c[4];
  site_coords(L, s, c);
  m3<double> K;
  for (int e = 0; e < 9; ++e) K.e[e] = {0, 0};
  for (int mu = 0; mu < 4; ++mu) {
    const double *plane = U + (int64_t)mu * 9 * V * 2;
    const int64_t sf = site_fwd(L, s, mu, c[mu]), sb = site_back(L, s, mu, c[mu]);
    m3<double> u, g, t;
    // U_mu(x) g^+(x+mu)
    for (int e = 0; e < 9; ++e) {
      u.e[e] = ldg(plane, (int64_t)e * V + s);
      g.e[e] = ldg(G, (int64_t)e * V + sf);
    }
    mul_adj(u, g, t);
    for (int e = 0; e < 9; ++e) K.e[e] = K.e[e] + t.e[e];
    // U_mu^+(x-mu) g^+(x-mu) = (g(x-mu) U_mu(x-mu))^+
    for (int e = 0; e < 9; ++e) {
      u.e[e] = ldg(plane, (int64_t)e * V + sb);
      g.e[e] = ldg(G, (int64_t)e * V + sb);
    }
    mul(g, u, t);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) K.e[3 * i + j] = K.e[3 * i + j] + conjg(t.e[3 * j + i]);
  }
  m3<double> W, M, Q, T1;
  for (int e = 0; e < 9; ++e) W.e[e] = ldg(Wp, (int64_t)e * V + s);
  double l[3];
  for (int k = 0; k < 3; ++k) l[k] = lam[(int64_t)k * V + s];
  // M = W^+ K W
  m3<double> Wd;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Wd.e[3 * i + j] = conjg(W.e[3 * j + i]);
  mul(Wd, K, T1);
  mul(T1, W, M);
  // Phi o M (Phi is symmetric)
  for (int j = 0; j < 3; ++j)
    for (int k = 0; k < 3; ++k) {
      double sn, cs;
      sincos(0.5 * (l[j] + l[k]), &sn, &cs);
      const double sc = sinc_half(0.5 * (l[j] - l[k]));
      M.e[3 * j + k] = M.e[3 * j + k] * cx<double>{cs * sc, sn * sc};
    }
  // Q = W (Phi o M) W^+
  mul(W, M, T1);
  mul_adj(T1, W, Q);
  // -(1/12V) Im Tr[T^a Q], T^a = lambda^a / 2
  const double f = -scale / (12.0 * (double)V);
  const double s3 = 0.57735026918962576451;
  double gr[8];
  gr[0] = 0.5 * (Q.e[3].i + Q.e[1].i);                       // lambda1: Q10 + Q01
  gr[1] = 0.5 * (-Q.e[3].r + Q.e[1].r);                      // lambda2: -i Q10 + i Q01
  gr[2] = 0.5 * (Q.e[0].i - Q.e[4].i);                       // lambda3
  gr[3] = 0.5 * (Q.e[6].i + Q.e[2].i);                       // lambda4: Q20 + Q02
  gr[4] = 0.5 * (-Q.e[6].r + Q.e[2].r);                      // lambda5
  gr[5] = 0.5 * (Q.e[7].i + Q.e[5].i);                       // lambda6: Q21 + Q12
  gr[6] = 0.5 * (-Q.e[7].r + Q.e[5].r);                      // lambda7
  gr[7] = 0.5 * s3 * (Q.e[0].i + Q.e[4].i - 2.0 * Q.e[8].i);  // lambda8
  for (int a = 0; a < 8; ++a) grad[s * 8 + a] = f * gr[a];
}

}  // namespace lgf
