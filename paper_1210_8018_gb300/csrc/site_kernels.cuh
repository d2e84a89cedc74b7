// site_kernels.cuh -- per-site kernels of one iteration of Algorithm 1 (Landau gauge fixing with
// Fourier acceleration): the Delta stencil with the theta/F reductions (Eqs. 1, 3-5), the formation
// of g (Eq. 2 to first order, then projection to SU(3)) and the gauge update of the links.
//
// Working layout (structure of arrays, one plane of V complex numbers per matrix element):
//   links  U[(mu*P + e)*V + s]   mu = 0..3, e = 3*row + col; P = 9 planes in double, P = 6 in float
//          (rows 0 and 1 only: the float stage is bound by memory traffic, so row 2 is rebuilt as
//          conj(row0 x row1) when a link is loaded -- the paper's "12 real" storage, Table 1)
//   g      G[e*V + s]; in the double path also a = g - 1 in double-float, A[e*V + s] as float4
//          (hi, lo of the real part, hi, lo of the imaginary part), read by the small-step update
//   packed Delta (and Delta-tilde) P[f*V + s], f = 0..3:
//     P0 = Delta_01, P1 = Delta_02, P2 = Delta_12, P3 = Im Delta_00 + i Im Delta_11.
//   Delta is anti-Hermitian and traceless, so these 8 reals determine it; the Fourier filter is real
//   and even in k, so it maps each packed field onto the packed field of the filtered matrix.
#pragma once
#include <type_traits>

#include "q61.cuh"
#include "su3.cuh"

namespace lgf {

struct Lattice {
  int n[4];         // Nx, Ny, Nz, Nt
  int64_t V;
  int64_t stride[4];  // 1, Nx, Nx*Ny, Nx*Ny*Nz
};

// Loop control shared by the kernels of the iteration, kept in device memory so that a sequence of
// iterations runs without host round trips.
struct Ctrl {
  double theta, F;       // values after the latest Delta evaluation
  double threshold;      // iterate while theta >= threshold
  double f_base;         // residual stage: F of the base links (F of the stage = f_base + residual part)
  int iters;             // gauge updates applied since load
  int limit;             // stop when iters reaches this
  int active;            // 1 while the loop runs; kernels return at once when 0
  int status;            // 0 ok, 5 non-finite theta or F
  unsigned int ticket;   // last-block counter of the reduction
  int hist_len;
  double *hist;          // device history: hist[2k], hist[2k+1] = theta, F after k updates
  unsigned int *ran;     // optional per-kernel counters of launches that did work (timing mode)
  int stage;             // precision of the live links: 0 float, 1 double, 2 the residual stage of the
                         // mixed schedule; kernels of another stage return at once (a batch launches
                         // the float and the double kernels in the mixed schedule)
  double plaq;           // average plaquette, written by k_plaquette
};
constexpr int kStageResidual = 2;

// Count a launch that does work (block 0, thread 0), for the per-kernel timing statistics.
__device__ __forceinline__ void count_run(const Ctrl *ctrl, int tkid) {
  if (ctrl->ran && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0)
    atomicAdd(ctrl->ran + tkid, 1u);
}

// Link storage: planes per link and the load/store of one link.
template <typename T> struct LinkStore {
  static constexpr int planes = 9;
};
template <> struct LinkStore<float> {
  static constexpr int planes = 6;
};
template <typename T> __device__ __forceinline__ void load_link(const T *plane, int64_t V, int64_t s, m3<T> &u) {
#pragma unroll
  for (int e = 0; e < LinkStore<T>::planes; ++e) u.e[e] = ldg(plane, (int64_t)e * V + s);
  if constexpr (LinkStore<T>::planes == 6) complete_row2(u);
}
// Store a link whose rows 0 and 1 are valid (row 2 is completed here when it is stored).
template <typename T> __device__ __forceinline__ void store_link(T *plane, int64_t V, int64_t s, m3<T> &u) {
  if constexpr (LinkStore<T>::planes == 9) complete_row2(u);
#pragma unroll
  for (int e = 0; e < LinkStore<T>::planes; ++e) st(plane, (int64_t)e * V + s, u.e[e]);
}
template <typename T> __device__ __forceinline__ int64_t link_plane_stride(int64_t V) {
  return (int64_t)LinkStore<T>::planes * V * 2;
}

// Batched launches: blockIdx.z selects one configuration of a group of equal-shape lattices whose
// buffers are stored one after the other; this is that configuration's loop control, and the
// kernel runs only if that configuration's loop is active in this kernel's precision.
template <typename T> __device__ __forceinline__ bool stage_active(const Ctrl *ctrl) {
  return ctrl->active && ctrl->stage == (sizeof(T) == 8 ? 1 : 0);
}
// check: 0 run unconditionally; 1 run if the loop is active in this kernel's precision; 2 run if the
// loop is active whatever the stage (a float FFT serving the double stage); 3 run if the loop is active
// in the residual stage (the float FFT of that stage).
template <typename T> __device__ __forceinline__ bool should_run(const Ctrl *ctrl, int check) {
  if (!check) return true;
  if (check == 3) return ctrl->active && ctrl->stage == kStageResidual;
  return check == 2 ? ctrl->active != 0 : stage_active<T>(ctrl);
}

__device__ __forceinline__ int64_t site_back(const Lattice &L, int64_t s, int mu, int c) {
  return c == 0 ? s + (int64_t)(L.n[mu] - 1) * L.stride[mu] : s - L.stride[mu];
}
__device__ __forceinline__ int64_t site_fwd(const Lattice &L, int64_t s, int mu, int c) {
  return c == L.n[mu] - 1 ? s - (int64_t)(L.n[mu] - 1) * L.stride[mu] : s + L.stride[mu];
}
// Coordinates of site s (V < 2^31 for every lattice that fits in memory, so 32-bit division).
__device__ __forceinline__ void site_coords(const Lattice &L, int64_t s64, int c[4]) {
  unsigned r = (unsigned)s64;
  c[0] = (int)(r % (unsigned)L.n[0]);
  r /= (unsigned)L.n[0];
  c[1] = (int)(r % (unsigned)L.n[1]);
  r /= (unsigned)L.n[1];
  c[2] = (int)(r % (unsigned)L.n[2]);
  c[3] = (int)(r / (unsigned)L.n[2]);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum a and b over the block (deterministic order); the result is valid in thread 0.
template <int NT> __device__ __forceinline__ void block_sum2(double &a, double &b) {
  __shared__ double sa[NT / 32], sb[NT / 32];
  a = warp_sum(a);
  b = warp_sum(b);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    sa[w] = a;
    sb[w] = b;
  }
  __syncthreads();
  if (w == 0) {
    a = l < NT / 32 ? sa[l] : 0.0;
    b = l < NT / 32 ? sb[l] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
  }
}

// Writes this block's (sum_theta, sum_F) partial; the last block to arrive reduces all partials in a
// fixed order and updates the loop control (Algorithm 1: "calculate Delta(x), F and theta", then the
// while-test theta >= eps). f_offset is added to F (the residual stage sums only the residual's traces).
// The block's number among the grid's nblk blocks is bid (blockIdx.x for one-dimensional grids).
template <int NT>
__device__ __forceinline__ void reduce_and_finalize_at(double th, double f, double *partials, Ctrl *ctrl, int64_t V,
                                                       int counts_update, double f_offset, unsigned bid,
                                                       unsigned nblk) {
  __shared__ bool last;
  block_sum2<NT>(th, f);
  if (threadIdx.x == 0) {
    partials[2 * bid] = th;
    partials[2 * bid + 1] = f;
    __threadfence();
    last = (atomicAdd(&ctrl->ticket, 1u) == nblk - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double a = 0.0, b = 0.0;
  for (unsigned k = threadIdx.x; k < nblk; k += NT) {
    a += __ldcg(partials + 2 * k);
    b += __ldcg(partials + 2 * k + 1);
  }
  __syncthreads();
  block_sum2<NT>(a, b);
  if (threadIdx.x == 0) {
    const double theta = a / (3.0 * (double)V);  // Eq. 4: 1/(N_c V) sum_x Tr[Delta Delta^+]
    const double F = b / (12.0 * (double)V) + f_offset;  // Eq. 1 at g = 1: 1/(4 N_c V) sum Re Tr U
    ctrl->ticket = 0;
    int it = ctrl->iters + counts_update;
    ctrl->iters = it;
    ctrl->theta = theta;
    ctrl->F = F;
    if (ctrl->hist && it < ctrl->hist_len) {
      ctrl->hist[2 * it] = theta;
      ctrl->hist[2 * it + 1] = F;
    }
    if (!isfinite(theta) || !isfinite(F)) {
      ctrl->status = 5;
      ctrl->active = 0;
    } else {
      ctrl->active = (theta >= ctrl->threshold) && (it < ctrl->limit);
    }
  }
}
template <int NT>
__device__ __forceinline__ void reduce_and_finalize(double th, double f, double *partials, Ctrl *ctrl, int64_t V,
                                                    int counts_update, double f_offset = 0.0) {
  reduce_and_finalize_at<NT>(th, f, partials, ctrl, V, counts_update, f_offset, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------------------------
// a1/a2: Delta(x) = sum_nu [U_nu(x-nu) - U_nu(x) - h.c. - trace] (Eqs. 3, 5), theta and F partials.
// Each thread handles kSitesPerThread sites (consecutive threads take consecutive sites). Only the
// nine real combinations that the anti-Hermitian traceless part needs are accumulated:
//   (B_01 - conj B_10), (B_02 - conj B_20), (B_12 - conj B_21) and Im B_00, Im B_11, Im B_22,
// with B = sum_nu [U_nu(x - nu) - U_nu(x)]. The per-site theta and F are formed in the kernel's
// precision and accumulated in double; the warp, block and global sums are double.
// ---------------------------------------------------------------------------------------------
constexpr int kSitesPerThread = 4;

template <typename T> __device__ __forceinline__ void accumulate_link(const m3<T> &u, T sign, T acc[9]) {
  acc[0] = fma(sign, u.e[1].r - u.e[3].r, acc[0]);
  acc[1] = fma(sign, u.e[1].i + u.e[3].i, acc[1]);
  acc[2] = fma(sign, u.e[2].r - u.e[6].r, acc[2]);
  acc[3] = fma(sign, u.e[2].i + u.e[6].i, acc[3]);
  acc[4] = fma(sign, u.e[5].r - u.e[7].r, acc[4]);
  acc[5] = fma(sign, u.e[5].i + u.e[7].i, acc[5]);
  acc[6] = fma(sign, u.e[0].i, acc[6]);
  acc[7] = fma(sign, u.e[4].i, acc[7]);
  acc[8] = fma(sign, u.e[8].i, acc[8]);
}

// The double path accumulates Delta in 64-bit fixed point with 56 fractional bits: Delta is a sum of
// eight O(1) link terms whose result is small, so integer sums give it exactly (up to the 2^-56
// quantisation of link entries below 2^-4, far below the FP64 rounding of the terms), and the integer
// pipe runs at 32 times the FP64 rate on this GPU. Converted back to double once, the result is at least
// as accurate as the FP64 sum. Entries of magnitude >= 64 (no unitary link has them) or non-finite
// entries set `bad`, which makes theta non-finite.
__device__ __forceinline__ long long q56(double x, bool &bad) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ed = (int)((b >> 52) & 0x7FF);
  bad |= ed > 1023 + 5;
  const unsigned long long m = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
  const int sh = ed - 1019;  // x * 2^56 = m * 2^(ed - 1075 + 56)
  unsigned long long q = sh >= 0 ? m << (sh & 15) : (sh > -64 ? m >> (-sh) : 0ull);
  if (ed == 0) q = 0ull;  // zero and subnormals
  const long long r = (long long)q;
  return (long long)b < 0 ? -r : r;
}
template <bool NEG> __device__ __forceinline__ void accumulate_link_q(const m3<double> &u, long long acc[9], bool &bad) {
  long long t[9];
  t[0] = q56(u.e[1].r, bad) - q56(u.e[3].r, bad);
  t[1] = q56(u.e[1].i, bad) + q56(u.e[3].i, bad);
  t[2] = q56(u.e[2].r, bad) - q56(u.e[6].r, bad);
  t[3] = q56(u.e[2].i, bad) + q56(u.e[6].i, bad);
  t[4] = q56(u.e[5].r, bad) - q56(u.e[7].r, bad);
  t[5] = q56(u.e[5].i, bad) + q56(u.e[7].i, bad);
  t[6] = q56(u.e[0].i, bad);
  t[7] = q56(u.e[4].i, bad);
  t[8] = q56(u.e[8].i, bad);
#pragma unroll
  for (int k = 0; k < 9; ++k) acc[k] = NEG ? acc[k] - t[k] : acc[k] + t[k];
}

// A float per-site value as a double by integer operations (the conversion instruction would occupy
// the FP64 pipe); doubles pass through.
__device__ __forceinline__ double widen_exact(float v) { return widen_bits(v); }
__device__ __forceinline__ double widen_exact(double v) { return v; }

// PT is the type of the packed output (T, or float when a double stage feeds a float FFT).
template <typename T, int NT, typename PT = T>
__device__ __forceinline__ void delta_body(const T *__restrict__ U, PT *__restrict__ P, double *partials, Ctrl *ctrl,
                                           Lattice L, int counts_update, int check_active, int tkid) {
  const int64_t V = L.V;
  {
    const int cfg = blockIdx.z;
    U += (int64_t)cfg * 4 * link_plane_stride<T>(V);
    P += (int64_t)cfg * 4 * V * 2;
    partials += (int64_t)cfg * 2 * gridDim.x;
    ctrl += cfg;
  }
  if (!should_run<T>(ctrl, check_active)) return;
  count_run(ctrl, tkid);
  double th = 0.0, f = 0.0;
  if constexpr (std::is_same<T, double>::value) {
#pragma unroll 1
    for (int k = 0; k < kSitesPerThread; ++k) {
      const int64_t s = ((int64_t)blockIdx.x * kSitesPerThread + k) * NT + threadIdx.x;
      if (s >= V) break;
      int c[4];
      site_coords(L, s, c);
      long long acc[9];
#pragma unroll
      for (int e = 0; e < 9; ++e) acc[e] = 0;
      bool bad = false;
      double fs = 0;
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) {
        const double *plane = U + (int64_t)mu * link_plane_stride<T>(V);
        m3<double> u;
        load_link(plane, V, site_back(L, s, mu, c[mu]), u);  // U_mu(x - mu)
        accumulate_link_q<false>(u, acc, bad);
        load_link(plane, V, s, u);  // - U_mu(x)
        accumulate_link_q<true>(u, acc, bad);
        fs += u.e[0].r + u.e[4].r + u.e[8].r;  // Re Tr U_mu(x)
      }
      constexpr double sc = 0x1p-56;
      double d[6];
#pragma unroll
      for (int e = 0; e < 6; ++e) d[e] = __ll2double_rn(acc[e]) * sc;
      // Delta_ii = 2i (Im B_ii - mean) = 2i (3 Im B_ii - sum) / 3
      const long long sd = acc[6] + acc[7] + acc[8];
      constexpr double w = 2.0 / 3.0 * sc;
      const double a0 = __ll2double_rn(3 * acc[6] - sd) * w, a1 = __ll2double_rn(3 * acc[7] - sd) * w;
      const double a2 = __ll2double_rn(3 * acc[8] - sd) * w;
      double ts = a0 * a0 + a1 * a1 + a2 * a2 +
                  2 * (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + d[3] * d[3] + d[4] * d[4] + d[5] * d[5]);
      if (bad) ts = __longlong_as_double(0x7FF8000000000000ll);  // non-finite or out-of-range link entries
      th += ts;
      f += fs;
      st(P, s, mkc(convert<PT>(d[0]), convert<PT>(d[1])));
      st(P, V + s, mkc(convert<PT>(d[2]), convert<PT>(d[3])));
      st(P, 2 * V + s, mkc(convert<PT>(d[4]), convert<PT>(d[5])));
      st(P, 3 * V + s, mkc(convert<PT>(a0), convert<PT>(a1)));
    }
  } else {
#pragma unroll 1
    for (int k = 0; k < kSitesPerThread; ++k) {
      const int64_t s = ((int64_t)blockIdx.x * kSitesPerThread + k) * NT + threadIdx.x;
      if (s >= V) break;
      int c[4];
      site_coords(L, s, c);
      T acc[9];
#pragma unroll
      for (int e = 0; e < 9; ++e) acc[e] = 0;
      T fs = 0;
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) {
        const T *plane = U + (int64_t)mu * link_plane_stride<T>(V);
        m3<T> u;
        load_link(plane, V, site_back(L, s, mu, c[mu]), u);  // U_mu(x - mu)
        accumulate_link(u, (T)1, acc);
        load_link(plane, V, s, u);  // - U_mu(x)
        accumulate_link(u, (T)-1, acc);
        fs += u.e[0].r + u.e[4].r + u.e[8].r;  // Re Tr U_mu(x)
      }
      // Delta_ij = acc (off-diagonal), Delta_ii = 2i (Im B_ii - mean)
      const T m = (acc[6] + acc[7] + acc[8]) / (T)3;
      const T a0 = 2 * (acc[6] - m), a1 = 2 * (acc[7] - m), a2 = 2 * (acc[8] - m);
      const T ts = a0 * a0 + a1 * a1 + a2 * a2 +
                   2 * (acc[0] * acc[0] + acc[1] * acc[1] + acc[2] * acc[2] + acc[3] * acc[3] + acc[4] * acc[4] +
                        acc[5] * acc[5]);
      th += widen_exact(ts);
      f += widen_exact(fs);
      st(P, s, mkc(convert<PT>(acc[0]), convert<PT>(acc[1])));
      st(P, V + s, mkc(convert<PT>(acc[2]), convert<PT>(acc[3])));
      st(P, 2 * V + s, mkc(convert<PT>(acc[4]), convert<PT>(acc[5])));
      st(P, 3 * V + s, mkc(convert<PT>(a0), convert<PT>(a1)));
    }
  }
  reduce_and_finalize<NT>(th, f, partials, ctrl, V, counts_update);
}

template <typename T, int NT, typename PT = T>
__global__ void __launch_bounds__(NT) k_delta(const T *__restrict__ U, PT *__restrict__ P, double *partials, Ctrl *ctrl,
                                             Lattice L, int counts_update, int check_active, int tkid) {
  delta_body<T, NT, PT>(U, P, partials, ctrl, L, counts_update, check_active, tkid);
}
// The float stage's Delta with five resident blocks per SM asked of the compiler (48 registers, 40 warps in
// flight instead of 32): the kernel waits on its link loads, and more warps hide that latency (measured at
// 64^4: 0.78 -> 0.71 ms per launch).
template <int NT>
__global__ void __launch_bounds__(NT, 5) k_delta_f32(const float *__restrict__ U, float *__restrict__ P,
                                                     double *partials, Ctrl *ctrl, Lattice L, int counts_update,
                                                     int check_active, int tkid) {
  delta_body<float, NT, float>(U, P, partials, ctrl, L, counts_update, check_active, tkid);
}

// The float Delta walking along t: thread (x, y, z) takes the TCH t-slices of chunk blockIdx.y, and the
// combinations of U_t(x) that it accumulates for one slice are those of the backward link U_t(x - t) of
// the next, kept in registers: seven links are read per site instead of eight. The same sums in the same
// order as delta_body (Delta is the same bits; theta and F partials are summed over other groups of sites).
// Measured at 64^4: 0.711 -> 0.649 ms per launch. Needs Nt % TCH == 0.
template <int NT, int TCH>
__global__ void __launch_bounds__(NT, 5) k_delta_f32_tw(const float *__restrict__ U, float *__restrict__ P,
                                                        double *partials, Ctrl *ctrl, Lattice L, int counts_update,
                                                        int check_active, int tkid) {
  const int64_t V = L.V;
  const unsigned nblk = gridDim.x * gridDim.y;
  {
    const int cfg = blockIdx.z;
    U += (int64_t)cfg * 4 * link_plane_stride<float>(V);
    P += (int64_t)cfg * 4 * V * 2;
    partials += (int64_t)cfg * 2 * nblk;
    ctrl += cfg;
  }
  if (!should_run<float>(ctrl, check_active)) return;
  count_run(ctrl, tkid);
  const int64_t nxyz = L.stride[3];
  const int64_t q = (int64_t)blockIdx.x * NT + threadIdx.x;
  double th = 0.0, f = 0.0;
  if (q < nxyz) {
    const int t0 = blockIdx.y * TCH;
    int c[4];
    site_coords(L, q + (int64_t)t0 * nxyz, c);
    const float *plane_t = U + 3 * link_plane_stride<float>(V);
    float tb[9];  // combinations of U_t(x - t): the previous slice's U_t(x)
    {
      m3<float> u;
      load_link(plane_t, V, site_back(L, q + (int64_t)t0 * nxyz, 3, t0), u);
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
        const float *plane = U + (int64_t)mu * link_plane_stride<float>(V);
        m3<float> u;
        load_link(plane, V, site_back(L, s, mu, c[mu]), u);  // U_mu(x - mu)
        accumulate_link(u, 1.f, acc);
        load_link(plane, V, s, u);  // - U_mu(x)
        accumulate_link(u, -1.f, acc);
        fs += u.e[0].r + u.e[4].r + u.e[8].r;  // Re Tr U_mu(x)
      }
      {
        m3<float> u;
        load_link(plane_t, V, s, u);
#pragma unroll
        for (int e = 0; e < 9; ++e) acc[e] = fmaf(1.f, tb[e], acc[e]);  // + U_t(x - t)
        accumulate_link(u, -1.f, acc);                                   // - U_t(x)
        fs += u.e[0].r + u.e[4].r + u.e[8].r;
#pragma unroll
        for (int e = 0; e < 9; ++e) tb[e] = 0.f;
        accumulate_link(u, 1.f, tb);
      }
      const float m = (acc[6] + acc[7] + acc[8]) / 3.f;
      const float a0 = 2 * (acc[6] - m), a1 = 2 * (acc[7] - m), a2 = 2 * (acc[8] - m);
      const float ts = a0 * a0 + a1 * a1 + a2 * a2 +
                       2 * (acc[0] * acc[0] + acc[1] * acc[1] + acc[2] * acc[2] + acc[3] * acc[3] +
                            acc[4] * acc[4] + acc[5] * acc[5]);
      th += widen_exact(ts);
      f += widen_exact(fs);
      st(P, s, mkc(acc[0], acc[1]));
      st(P, V + s, mkc(acc[2], acc[3]));
      st(P, 2 * V + s, mkc(acc[4], acc[5]));
      st(P, 3 * V + s, mkc(a0, a1));
    }
  }
  reduce_and_finalize_at<NT>(th, f, partials, ctrl, V, counts_update, 0.0, blockIdx.x + gridDim.x * blockIdx.y, nblk);
}

// Rebuild the full anti-Hermitian traceless matrix from the packed fields (type PT), scaled by a.
template <typename T, typename PT = T>
__device__ __forceinline__ void unpack_scaled(const PT *P, int64_t V, int64_t s, T a, m3<T> &m) {
  const cx<PT> q0 = ldg(P, s), q1 = ldg(P, V + s), q2 = ldg(P, 2 * V + s), q3 = ldg(P, 3 * V + s);
  const cx<T> p0 = {convert<T>(q0.r), convert<T>(q0.i)}, p1 = {convert<T>(q1.r), convert<T>(q1.i)};
  const cx<T> p2 = {convert<T>(q2.r), convert<T>(q2.i)}, p3 = {convert<T>(q3.r), convert<T>(q3.i)};
  const T zero = kconst<T>(0.0);
  m.e[0] = {zero, a * p3.r};
  m.e[4] = {zero, a * p3.i};
  m.e[8] = {zero, -a * (p3.r + p3.i)};
  m.e[1] = scale(p0, a);
  m.e[2] = scale(p1, a);
  m.e[5] = scale(p2, a);
  m.e[3] = {-a * p0.r, a * p0.i};  // -conj(a p0)
  m.e[6] = {-a * p1.r, a * p1.i};
  m.e[7] = {-a * p2.r, a * p2.i};
}

// ---------------------------------------------------------------------------------------------
// a6: g(x) = SU(3)-projection of [1 + (alpha/2) Delta-tilde(x)] (Eq. 2 expanded to first order in
// alpha, then reunitarized).
// ---------------------------------------------------------------------------------------------
//
// Small-step form of the projection (double path): with X = (alpha/2) Delta-tilde small, Gram-Schmidt of
// 1 + X is written as g = 1 + a, and a is formed from small quantities only, in double-float:
//   row 0: |e0 + x0|^2 = 1 + t0, t0 = 2 Re x0_0 + |x0|^2; a0 = x0 (1 + c0) + c0 e0 with
//          c0 = (1 + t0)^(-1/2) - 1;
//   row 1: p = <g0, e1 + x1> = conj(a0_1) + x1_0 + sum_j conj(a0_j) x1_j; d1 = x1 - p (e0 + a0);
//          |e1 + d1|^2 = 1 + t1, t1 = 2 Re d1_1 + |d1|^2; a1 = d1 (1 + c1) + c1 e1;
//   row 2: conj(g0 x g1) - e2 = conj(e0 x a1 + a0 x e1 + a0 x a1).
// (1 + t)^(-1/2) - 1 is the series -t/2 + 3t^2/8 - 5t^3/16, whose remainder is below 2^-54 for
// |t| <= 2^-13. When every element of X is below 2^-8 in magnitude, a has an absolute error of a few
// 2^-48 |a|, below the FP64 rounding of g, and g = 1 + a is assembled in FP64.
constexpr int kSmallXFloatExpField = 127 - 9;  // |x| < 2^-8  <=>  float exponent field <= 118

__device__ __forceinline__ int fexp_field(float x) { return (int)((__float_as_uint(x) >> 23) & 0xFF); }
template <typename T> __device__ __forceinline__ T rsqrt1p_m1(T t) {
  return t * (kconst<T>(-0.5) + t * (kconst<T>(0.375) + t * kconst<T>(-0.3125)));
}
// (T = df64 for the double path; T = float for the residual stage of the mixed schedule)
template <typename T> __device__ __forceinline__ void small_step_projection(const m3<T> &X, m3<T> &a) {
  const T one = kconst<T>(1.0);
  const T t0 = kconst<T>(2.0) * X.e[0].r + (norm2(X.e[0]) + norm2(X.e[1]) + norm2(X.e[2]));
  const T c0 = rsqrt1p_m1(t0), s0 = one + c0;
  a.e[0] = scale(X.e[0], s0) + cx<T>{c0, kconst<T>(0.0)};
  a.e[1] = scale(X.e[1], s0);
  a.e[2] = scale(X.e[2], s0);
  cx<T> p = conjg(a.e[1]) + X.e[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) p = p + conjg(a.e[j]) * X.e[3 + j];
  cx<T> d[3];
  d[0] = X.e[3] - p - p * a.e[0];
  d[1] = X.e[4] - p * a.e[1];
  d[2] = X.e[5] - p * a.e[2];
  const T t1 = kconst<T>(2.0) * d[1].r + (norm2(d[0]) + norm2(d[1]) + norm2(d[2]));
  const T c1 = rsqrt1p_m1(t1), s1 = one + c1;
  a.e[3] = scale(d[0], s1);
  a.e[4] = scale(d[1], s1) + cx<T>{c1, kconst<T>(0.0)};
  a.e[5] = scale(d[2], s1);
  a.e[6] = conjg(a.e[1] * a.e[5] - a.e[2] * a.e[4] - a.e[2]);
  a.e[7] = conjg(a.e[2] * a.e[3] - a.e[0] * a.e[5] - a.e[5]);
  a.e[8] = conjg(a.e[0] * a.e[4] - a.e[1] * a.e[3] + a.e[4] + a.e[0]);
}

// The double path also stores a = g - 1 in double-float (A, 9 planes of float4): the small-step update
// reads a and its neighbours' b = g(x+mu) - 1 from there without conversions.
__device__ __forceinline__ void st_a(float *A, int64_t idx, cx<df64> v) {
  reinterpret_cast<float4 *>(A)[idx] = to_vec<df64>(v);
}
__device__ __forceinline__ cx<df64> minus_identity_split(cx<double> v, int e) {
  if (e == 0 || e == 4 || e == 8) v.r -= 1.0;  // exact for |g_ii - 1| <= 1/2 (Sterbenz)
  return {df64_split_fast(v.r), df64_split_fast(v.i)};
}

template <typename T, int NT, typename PT = T>
__global__ void __launch_bounds__(NT) k_gauge(const PT *__restrict__ P, T *__restrict__ G, float *__restrict__ A,
                                             T half_alpha, int64_t V, const Ctrl *ctrl, int check_active, int tkid,
                                             int allow_small) {
  {
    const int cfg = blockIdx.z;
    P += (int64_t)cfg * 4 * V * 2;
    G += (int64_t)cfg * 9 * V * 2;
    if (A) A += (int64_t)cfg * 9 * V * 4;
    ctrl += cfg;
  }
  if (!should_run<T>(ctrl, check_active)) return;
  count_run(ctrl, tkid);
  const int64_t s = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (s >= V) return;
  if constexpr (std::is_same<T, double>::value) {
    m3<df64> X;
    unpack_scaled<df64, PT>(P, V, s, convert<df64>(half_alpha), X);
    int ef = 0;
#pragma unroll
    for (int e = 0; e < 9; ++e) ef = max(ef, max(fexp_field(X.e[e].r.hi), fexp_field(X.e[e].i.hi)));
    if (__all_sync(__activemask(), allow_small && ef <= kSmallXFloatExpField)) {
      m3<df64> a;
      small_step_projection(X, a);
#pragma unroll
      for (int e = 0; e < 9; ++e) {
        double re = convert<double>(a.e[e].r);
        if (e == 0 || e == 4 || e == 8) re = 1.0 + re;
        st(G, (int64_t)e * V + s, mkc(re, convert<double>(a.e[e].i)));
        if (A) st_a(A, (int64_t)e * V + s, a.e[e]);
      }
      return;
    }
  }
  m3<T> g;
  unpack_scaled<T, PT>(P, V, s, half_alpha, g);
  g.e[0].r += 1;
  g.e[4].r += 1;
  g.e[8].r += 1;
  reunitarize(g);
#pragma unroll
  for (int e = 0; e < 9; ++e) st(G, (int64_t)e * V + s, g.e[e]);
  if constexpr (std::is_same<T, double>::value) {
    if (A) {
#pragma unroll
      for (int e = 0; e < 9; ++e) st_a(A, (int64_t)e * V + s, minus_identity_split(g.e[e], e));
    }
  }
}

// A = g - 1 in double-float from a g field (the single-step update takes g from the caller).
template <int NT> __global__ void k_a_from_g(const double *__restrict__ G, float *__restrict__ A, int64_t V) {
  const int64_t s = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (s >= V) return;
#pragma unroll
  for (int e = 0; e < 9; ++e) st_a(A, (int64_t)e * V + s, minus_identity_split(ldg(G, (int64_t)e * V + s), e));
}

// ---------------------------------------------------------------------------------------------
// a7: U_mu(x) -> g(x) U_mu(x) g^dagger(x + mu) for the four directions.
//
// Double links take one of two forms of the same product, chosen per warp and per link:
//  * small step: with g(x) = 1 + a and g(x+mu) = 1 + b, rows 0 and 1 of the new link are U + delta with
//      delta = a U + (U + a U) b^dagger,
//    delta formed in double-float arithmetic (FP32 operations, ~2^-48 relative) and added to U in
//    FP64; row 2 = conj(row0 x row1) in FP64. When every element of a and b is below 2^-7 in magnitude, delta's absolute error (a few
//    2^-48 |a| |U|) is at or below the FP64 rounding of the product itself, and the FP64 pipe -- 1/64
//    of the FP32 rate on this GPU -- does only the final additions. Near convergence |a| ~ alpha |Delta|
//    is far below the bound.
//  * general step: rows 0 and 1 of g(x) U g^+(x+mu) by FP64 products, row 2 = conj(row0 x row1).
// ---------------------------------------------------------------------------------------------
constexpr int kSmallStepFloatExpField = 127 - 8;  // |x| < 2^-7  <=>  float exponent field of hi <= 119

// Largest float exponent field of the high parts of a double-float complex element, with the running max.
__device__ __forceinline__ int exp_max_df(cx<df64> v, int emax) {
  return max(emax, max((int)((__float_as_uint(v.r.hi) >> 23) & 0xFF), (int)((__float_as_uint(v.i.hi) >> 23) & 0xFF)));
}
__device__ __forceinline__ cx<df64> dfc_add(cx<df64> x, cx<df64> y) { return {x.r + y.r, x.i + y.i}; }
// (integer widening: the float -> double conversion instruction occupies the FP64 pipe)
__device__ __forceinline__ double df64_widen(df64 x) { return widen_bits(x.hi) + widen_bits(x.lo); }

// Asynchronous 16-byte global -> shared copies (each thread copies, and later reads, only its own slots,
// so completing its own groups is all the ordering needed).
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Shared memory of the double update per block of NT threads, [slot][thread] in 16-byte units:
// a = g(x) - 1 (9 slots), the link (9), b = g(x+mu) - 1 (9), a and b in double-float: 432 B per thread,
// so that four blocks of 128 threads (16 warps) fit on an SM.
template <int NT> constexpr size_t update_smem_bytes() { return (size_t)27 * NT * 16; }

template <int NT>
__device__ __forceinline__ void fetch_u(const double *plane, int64_t V, int64_t s, double2 *bu) {
  const double2 *pu = reinterpret_cast<const double2 *>(plane);
#pragma unroll
  for (int e = 0; e < 9; ++e) cp_async16(bu + e * NT + threadIdx.x, pu + (int64_t)e * V + s);
  cp_async_commit();
}
template <int NT>
__device__ __forceinline__ void fetch_b(const float *A, int64_t V, int64_t sf, float4 *bb) {
  const float4 *pa = reinterpret_cast<const float4 *>(A);
#pragma unroll
  for (int e = 0; e < 9; ++e) cp_async16(bb + e * NT + threadIdx.x, pa + (int64_t)e * V + sf);
  cp_async_commit();
}
// Start the copies of link mu at site s (9 elements to bu) and of b at its forward neighbour sf (to bb).
template <int NT>
__device__ __forceinline__ void fetch_link(const double *plane, const float *A, int64_t V, int64_t s, int64_t sf,
                                           double2 *bu, float4 *bb) {
  const double2 *pu = reinterpret_cast<const double2 *>(plane);
  const float4 *pa = reinterpret_cast<const float4 *>(A);
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    cp_async16(bu + e * NT + threadIdx.x, pu + (int64_t)e * V + s);
    cp_async16(bb + e * NT + threadIdx.x, pa + (int64_t)e * V + sf);
  }
  cp_async_commit();
}

// Small-step update of one link: u (the link) and b = g(x+mu) - 1 in double-float registers, a (rows of
// g(x) - 1) in shared memory, the FP64 link in bu; the new link is stored to the plane.
template <int NT>
__device__ __forceinline__ void update_link_small(double *plane, int64_t V, int64_t s, const float4 *sa,
                                                  double2 *bu, const cx<df64> u[9], const cx<df64> b[9]) {
  // rows 0 and 1 one at a time (a rolled loop keeps the code within the instruction cache); each new
  // element replaces the old one in bu
#pragma unroll 1
  for (int i = 0; i < 2; ++i) {
    cx<df64> ai[3], ui[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      ai[k] = from_vec<df64>(sa[(3 * i + k) * NT + threadIdx.x]);
      ui[k] = i == 0 ? u[k] : u[3 + k];
    }
    cx<df64> v[3], y[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {  // v = row i of a U
      dfacc re = dfacc_prod(ai[0].r, u[j].r), im = dfacc_prod(ai[0].r, u[j].i);
      dfacc_msub(re, ai[0].i, u[j].i);
      dfacc_mac(im, ai[0].i, u[j].r);
#pragma unroll
      for (int k = 1; k < 3; ++k) {
        dfacc_mac(re, ai[k].r, u[3 * k + j].r);
        dfacc_msub(re, ai[k].i, u[3 * k + j].i);
        dfacc_mac(im, ai[k].r, u[3 * k + j].i);
        dfacc_mac(im, ai[k].i, u[3 * k + j].r);
      }
      v[j] = {dfacc_result(re), dfacc_result(im)};
      y[j] = dfc_add(ui[j], v[j]);
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {  // delta_ij = v_j + sum_k y_k conj(b_jk); new U_ij = U_ij + delta_ij
      dfacc re = dfacc_from(v[j].r), im = dfacc_from(v[j].i);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        dfacc_mac(re, y[k].r, b[3 * j + k].r);
        dfacc_mac(re, y[k].i, b[3 * j + k].i);
        dfacc_mac(im, y[k].i, b[3 * j + k].r);
        dfacc_msub(im, y[k].r, b[3 * j + k].i);
      }
      const int e = 3 * i + j;
      const double2 old = bu[e * NT + threadIdx.x];
      const double2 nu = make_double2(old.x + df64_widen(dfacc_result(re)), old.y + df64_widen(dfacc_result(im)));
      bu[e * NT + threadIdx.x] = nu;
      st(plane, (int64_t)e * V + s, from_vec<double>(nu));
    }
  }
  // row 2 = conj(row0 x row1) in FP64, as in the general form (the FP64 pipe has room here)
  cx<double> r0[3], r1[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    r0[j] = from_vec<double>(bu[j * NT + threadIdx.x]);
    r1[j] = from_vec<double>(bu[(3 + j) * NT + threadIdx.x]);
  }
  st(plane, 6 * V + s, cross_cj(r0[1], r1[2], r0[2], r1[1]));
  st(plane, 7 * V + s, cross_cj(r0[2], r1[0], r0[0], r1[2]));
  st(plane, 8 * V + s, cross_cj(r0[0], r1[1], r0[1], r1[0]));
}

// General-step update of one link in FP64: rows 0 and 1 of g(x) U g^+(x+mu) by products (g(x) and
// g(x+mu) from global memory, the link from bu), row 2 = conj(row0 x row1).
template <int NT>
__device__ __forceinline__ void update_link_general(double *plane, const double *G, int64_t V, int64_t s,
                                                    int64_t sf, const double2 *bu) {
  m3<double> t;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    cx<double> gi[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) gi[k] = ldg(G, (int64_t)(3 * i + k) * V + s);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cx<double> acc = gi[0] * from_vec<double>(bu[j * NT + threadIdx.x]);
      acc = cmac(acc, gi[1], from_vec<double>(bu[(3 + j) * NT + threadIdx.x]));
      acc = cmac(acc, gi[2], from_vec<double>(bu[(6 + j) * NT + threadIdx.x]));
      t.e[3 * i + j] = acc;
    }
  }
  m3<double> o;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const cx<double> h0 = ldg(G, (int64_t)(3 * j) * V + sf);
    const cx<double> h1 = ldg(G, (int64_t)(3 * j + 1) * V + sf);
    const cx<double> h2 = ldg(G, (int64_t)(3 * j + 2) * V + sf);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      cx<double> acc = {0, 0};
      acc = cmac_cj(acc, t.e[3 * i], h0);
      acc = cmac_cj(acc, t.e[3 * i + 1], h1);
      acc = cmac_cj(acc, t.e[3 * i + 2], h2);
      o.e[3 * i + j] = acc;
    }
  }
  store_link(plane, V, s, o);
}

// The same general-step product in 61-bit fixed point (q61.cuh) on the integer pipe: rows 0 and 1 of
// g(x) U g^+(x+mu) exact to FP64 rounding, row 2 = conj(row0 x row1) in fixed point.
template <int NT>
__device__ __forceinline__ void update_link_general_q(double *plane, const double *G, int64_t V, int64_t s,
                                                      int64_t sf, const double2 *bu) {
  cq t[6];
  {
    cq gx[6];
#pragma unroll
    for (int e = 0; e < 6; ++e) gx[e] = to_cq(ldg(G, (int64_t)e * V + s));
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const cq u0 = to_cq(from_vec<double>(bu[j * NT + threadIdx.x]));
      const cq u1 = to_cq(from_vec<double>(bu[(3 + j) * NT + threadIdx.x]));
      const cq u2 = to_cq(from_vec<double>(bu[(6 + j) * NT + threadIdx.x]));
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        cq a = {0, 0};
        cq_mac(a, gx[3 * i], u0);
        cq_mac(a, gx[3 * i + 1], u1);
        cq_mac(a, gx[3 * i + 2], u2);
        t[3 * i + j] = a;
      }
    }
  }
  cq o[9];
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
  for (int e = 0; e < 9; ++e) st(plane, (int64_t)e * V + s, cx<double>{from_q61(o[e].r), from_q61(o[e].i)});
}

// Double links: general steps are split between the FP64 pipe (the first fp64_even or fp64_odd directions
// of a site, in even or odd warps) and the integer pipe (the others, in Q61), so that both pipes work at the
// same time; both forms are exact to FP64 rounding.
template <typename T, int NT>
__global__ void __launch_bounds__(NT, sizeof(T) == 8 ? 4 : 2)
    k_update(T *__restrict__ U, const T *__restrict__ G, const float *__restrict__ A, Lattice L, const Ctrl *ctrl,
             int check_active, int tkid, int allow_small, int fp64_even, int fp64_odd) {
  const int64_t V = L.V;
  {
    const int cfg = blockIdx.z;
    U += (int64_t)cfg * 4 * link_plane_stride<T>(V);
    G += (int64_t)cfg * 9 * V * 2;
    if (A) A += (int64_t)cfg * 9 * V * 4;
    ctrl += cfg;
  }
  if (!should_run<T>(ctrl, check_active)) return;
  count_run(ctrl, tkid);
  const int64_t s = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (s >= V) return;
  int c[4];
  site_coords(L, s, c);
  if constexpr (std::is_same<T, double>::value) {
    // b of link mu + 1 is copied while link mu is computed, the link itself once link mu is stored
    // (dynamic shared memory of update_smem_bytes<NT>()); 16 resident warps cover that latency.
    extern __shared__ __align__(16) unsigned char update_smem[];
    float4 *sa = reinterpret_cast<float4 *>(update_smem);
    double2 *bu0 = reinterpret_cast<double2 *>(sa + 9 * NT);
    float4 *bb = reinterpret_cast<float4 *>(bu0 + 9 * NT);
    const int64_t pstride = link_plane_stride<T>(V);
    {  // a = g(x) - 1 with the first link and b (one group of copies)
      const float4 *pa = reinterpret_cast<const float4 *>(A);
#pragma unroll
      for (int e = 0; e < 9; ++e) cp_async16(sa + e * NT + threadIdx.x, pa + (int64_t)e * V + s);
    }
    fetch_link<NT>(U, A, V, s, site_fwd(L, s, 0, c[0]), bu0, bb);
    cp_async_wait_all();
    int ea = 0;
#pragma unroll
    for (int e = 0; e < 9; ++e) ea = exp_max_df(from_vec<df64>(sa[e * NT + threadIdx.x]), ea);
#pragma unroll 1
    for (int mu = 0; mu < 4; ++mu) {
      double *plane = U + (int64_t)mu * pstride;
      const double2 *bu = bu0;
      cp_async_wait_all();
      cx<df64> b[9];
      int eb = ea;
#pragma unroll
      for (int e = 0; e < 9; ++e) {
        b[e] = from_vec<df64>(bb[e * NT + threadIdx.x]);
        eb = exp_max_df(b[e], eb);
      }
      const int64_t sf = site_fwd(L, s, mu, c[mu]);
      if (__all_sync(__activemask(), allow_small && eb <= kSmallStepFloatExpField)) {
        cx<df64> u[9];
#pragma unroll
        for (int e = 0; e < 9; ++e) {
          const double2 v = bu[e * NT + threadIdx.x];
          u[e] = {df64_split_fast(v.x), df64_split_fast(v.y)};
        }
        if (mu < 3) fetch_b<NT>(A, V, site_fwd(L, s, mu + 1, c[mu + 1]), bb);
        update_link_small<NT>(plane, V, s, sa, bu0, u, b);
        if (mu < 3) fetch_u<NT>(plane + pstride, V, s, bu0);
      } else {
        const int nf = ((threadIdx.x >> 5) & 1) ? fp64_odd : fp64_even;  // uniform within a warp
        if (mu < nf) update_link_general<NT>(plane, G, V, s, sf, bu);
        else update_link_general_q<NT>(plane, G, V, s, sf, bu);
        if (mu < 3) fetch_link<NT>(plane + pstride, A, V, s, site_fwd(L, s, mu + 1, c[mu + 1]), bu0, bb);
      }
    }
  } else {
    m3<T> gx;
#pragma unroll
    for (int e = 0; e < 9; ++e) gx.e[e] = ldg(G, (int64_t)e * V + s);
#pragma unroll 1
    for (int mu = 0; mu < 4; ++mu) {
      const int64_t sf = site_fwd(L, s, mu, c[mu]);
      T *plane = U + (int64_t)mu * link_plane_stride<T>(V);
      m3<T> u, gy, t;
      load_link(plane, V, s, u);
#pragma unroll
      for (int e = 0; e < 9; ++e) gy.e[e] = ldg(G, (int64_t)e * V + sf);
      // rows 0 and 1 of g(x) U g^+(x+mu) by products, row 2 = conj(row0 x row1) (the result is in SU(3))
      mul_rows01(gx, u, t);
      mul_adj_rows01(t, gy, u);
      store_link(plane, V, s, u);
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Layout conversions between the caller's array-of-structures links / site fields (double) and the
// working planes (T). These run once per load/store, not in the loop.
// ---------------------------------------------------------------------------------------------
// A: nmat*V matrices of 9 complex; Pl: planes [(m*np + e)*V + s], np = 9, or 6 (rows 0-1 of links). The
// launch converts the matrices idx0 .. idx0 + n - 1 (a chunk, when the copy from the host is pipelined).
template <typename T>
__global__ void k_aos_to_planes(const double *__restrict__ A, T *__restrict__ Pl, int64_t V, int nmat, int np,
                                int64_t idx0, int64_t n) {
  const int64_t idx = idx0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= idx0 + n || idx >= (int64_t)nmat * V) return;
  const int64_t m = idx / V, s = idx - m * V;
  const double2 *src = reinterpret_cast<const double2 *>(A) + idx * 9;
  for (int e = 0; e < np; ++e) {
    const double2 v = src[e];
    st(Pl, (m * np + e) * V + s, mkc((T)v.x, (T)v.y));
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_planes_to_aos(const T *__restrict__ Pl, double *__restrict__ A, int64_t V,
                                                       int nmat, int np, int64_t idx0, int64_t n) {
  // Each thread forms one matrix from the planes (coalesced loads) into shared memory; the block then
  // writes its matrices' contiguous 144-byte records with consecutive threads on consecutive 16-byte
  // chunks (a thread writing its own record would put every store instruction's 32 chunks 144 bytes apart).
  constexpr int NTB = 256;
  __shared__ double2 rec[NTB * 9];
  const int64_t first = idx0 + (int64_t)blockIdx.x * NTB;
  const int64_t end = min(idx0 + n, (int64_t)nmat * V);
  const int cnt = (int)max((int64_t)0, min((int64_t)NTB, end - first));
  const int64_t idx = first + threadIdx.x;
  if (threadIdx.x < cnt) {
    const int64_t m = idx / V, s = idx - m * V;
    m3<T> u;
    for (int e = 0; e < np; ++e) u.e[e] = ld(Pl, (m * np + e) * V + s);
    if (np == 6) complete_row2(u);
#pragma unroll
    for (int e = 0; e < 9; ++e) rec[threadIdx.x * 9 + e] = make_double2((double)u.e[e].r, (double)u.e[e].i);
  }
  __syncthreads();
  double2 *dst = reinterpret_cast<double2 *>(A) + first * 9;
  for (int q = threadIdx.x; q < cnt * 9; q += NTB) dst[q] = rec[q];
}

// Full site matrices (AoS double) <-> packed anti-Hermitian traceless fields (planes of PT).
template <typename PT> __global__ void k_pack_antiherm(const double *__restrict__ A, PT *__restrict__ P, int64_t V) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  const double2 *m = reinterpret_cast<const double2 *>(A) + s * 9;
  st(P, s, mkc(convert<PT>(m[1].x), convert<PT>(m[1].y)));
  st(P, V + s, mkc(convert<PT>(m[2].x), convert<PT>(m[2].y)));
  st(P, 2 * V + s, mkc(convert<PT>(m[5].x), convert<PT>(m[5].y)));
  st(P, 3 * V + s, mkc(convert<PT>(m[0].y), convert<PT>(m[4].y)));
}

template <typename PT> __global__ void k_unpack_antiherm(const PT *__restrict__ P, double *__restrict__ A, int64_t V) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  using T = typename std::conditional<sizeof(PT) == 4, float, double>::type;
  m3<T> m;
  unpack_scaled<T, PT>(P, V, s, (T)1, m);
  double2 *dst = reinterpret_cast<double2 *>(A) + s * 9;
#pragma unroll
  for (int e = 0; e < 9; ++e) dst[e] = make_double2((double)m.e[e].r, (double)m.e[e].i);
}

// The eight real coefficient fields of an su(3) field, c^a(s) = coef[8 s + a], held as the four complex
// fields c^(2j) + i c^(2j+1), j = 0..3, in the packed planes: the Fourier filter of Algorithm 1 is real and
// even in k, so it maps the real and the imaginary part of each plane separately, and the planes come back
// as the four pairs of filtered coefficient fields.
template <typename PT> __global__ void k_pack_coeffs(const double *__restrict__ c, PT *__restrict__ P, int64_t V) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  const double2 *q = reinterpret_cast<const double2 *>(c) + s * 4;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const double2 v = q[j];
    st(P, (int64_t)j * V + s, mkc(convert<PT>(v.x), convert<PT>(v.y)));
  }
}

template <typename PT> __global__ void k_unpack_coeffs(const PT *__restrict__ P, double *__restrict__ c, int64_t V) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  double2 *q = reinterpret_cast<double2 *>(c) + s * 4;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const cx<PT> v = ldg(P, (int64_t)j * V + s);
    q[j] = make_double2(convert<double>(v.r), convert<double>(v.i));
  }
}

// Average plaquette partials: (1/3) Re Tr U_mu(x) U_nu(x+mu) U_mu^+(x+nu) U_nu^+(x) over mu < nu.
template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_plaquette(const T *__restrict__ U, double *partials, Ctrl *ctrl, Lattice L) {
  const int64_t V = L.V;
  double acc = 0.0;
  for (int k = 0; k < kSitesPerThread; ++k) {
    const int64_t s = ((int64_t)blockIdx.x * kSitesPerThread + k) * NT + threadIdx.x;
    if (s >= V) break;
    int c[4];
    site_coords(L, s, c);
    for (int mu = 0; mu < 4; ++mu)
      for (int nu = mu + 1; nu < 4; ++nu) {
        const int64_t smu = site_fwd(L, s, mu, c[mu]), snu = site_fwd(L, s, nu, c[nu]);
        m3<T> a, b, t, w;
        for (int e = 0; e < 9; ++e) {
          a.e[e] = ldg(U + (int64_t)mu * 9 * V * 2, (int64_t)e * V + s);
          b.e[e] = ldg(U + (int64_t)nu * 9 * V * 2, (int64_t)e * V + smu);
        }
        mul(a, b, t);  // U_mu(x) U_nu(x+mu)
        for (int e = 0; e < 9; ++e) {
          a.e[e] = ldg(U + (int64_t)mu * 9 * V * 2, (int64_t)e * V + snu);
          b.e[e] = ldg(U + (int64_t)nu * 9 * V * 2, (int64_t)e * V + s);
        }
        mul(b, a, w);  // U_nu(x) U_mu(x+nu)
        // Re Tr[t w^+] = sum_ij Re t_ij conj(w_ij)
        for (int e = 0; e < 9; ++e) acc += (double)t.e[e].r * w.e[e].r + (double)t.e[e].i * w.e[e].i;
      }
  }
  // block sums, then the last block to finish sums the partials in block order (as for theta and F)
  __shared__ bool last;
  double dummy = 0.0;
  block_sum2<NT>(acc, dummy);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = acc;
    __threadfence();
    last = (atomicAdd(&ctrl->ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double a = 0.0, b = 0.0;
  for (unsigned k = threadIdx.x; k < gridDim.x; k += NT) a += __ldcg(partials + k);
  __syncthreads();
  block_sum2<NT>(a, b);
  if (threadIdx.x == 0) {
    ctrl->plaq = a / (3.0 * 6.0 * (double)V);  // (1/3) Re Tr over V sites and 6 planes
    ctrl->ticket = 0;
  }
}

}  // namespace lgf
