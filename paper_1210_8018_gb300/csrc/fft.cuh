// fft.cuh -- hand-written batched 4D FFT with the Fourier-acceleration filter of Algorithm 1.
//
// Each packed Delta field (4 per site, see site_kernels.cuh) is transformed by a sequence of
// "passes". A pass stages a tile of the field in shared memory -- the full extent of one or two
// lattice axes times a run of C elements that are contiguous in memory -- transforms the tile along
// those axes and writes it back. The forward transform is an in-place mixed-radix decimation-in-
// frequency FFT, which leaves the spectrum in digit-reversed order; the filter reads the frequency of
// each position from tables, and the inverse runs the exact inverse stages (decimation in time) in
// reverse order, which restores natural order. No permutation pass is needed. The filter
// w(k) = p^2_max / (V p^2(k)), w(0) = 0, is applied inside the last forward pass, which then runs the
// inverse along its own axes before writing (Algorithm 1: FFT forward, p^2_max/p^2, FFT backward,
// normalize).
//
// DIF stage (block length L, radix R, M = L/R), for each block and each j in [0, M):
//   y_r' = w_L^{j r'} * sum_r x[j + M r] w_R^{r r'},   stored at j + M r',   w_n = exp(-2 pi i / n).
// The inverse stage undoes it exactly up to the factor R.
#pragma once
#include "site_kernels.cuh"

namespace lgf {

constexpr int kMaxStages = 8;

struct AxisFFT {
  int N;                  // axis length
  int nst;                // number of stages
  int R[kMaxStages];      // radix of each DIF stage, in forward order
};

// One pass: a tile of extents d[0] (fastest in shared memory) x d[1] x d[2]; tile element
// (i0, i1, i2) lives at global complex index base(b) + i0*g[0] + i1*g[1] + i2*g[2] of a field, with
// base(b) = (b % nb1)*B1 + (b / nb1)*B2 for block b. The pass transforms along nax tile dimensions.
struct PassDesc {
  int d[3];
  int64_t g[3];
  int nb1;
  int64_t B1, B2;
  int nax;
  int ax_dim[2];   // tile dimension of each transformed axis
  int ax_mu[2];    // lattice axis (0..3) of each
  int mode;        // 0 forward, 1 inverse, 2 forward + filter + inverse
  int nblocks;     // blocks per field
};

struct FFTTables {
  AxisFFT ax[4];
  const void *tw[4];        // per lattice axis: N complex twiddles w_N^j (T)
  const double *p2part[4];  // per lattice axis: 4 sin^2(pi k(pos)/N) for the frequency at position pos
  double wscale;            // p^2_max / V
  int n[4];
};

// Butterfly sums. In double-float the pair is not renormalised after each addition (TwoSum of the high
// parts plus the low parts: 8 operations instead of 11); the twiddle multiplication renormalises, so the
// low part grows by at most a few ulps of the high part between multiplications. The transform's error
// stays ~2^-45 of the field norm, far below what the filter (which only sets the step direction) needs.
template <typename T> __device__ __forceinline__ cx<T> badd(cx<T> a, cx<T> b) { return a + b; }
template <typename T> __device__ __forceinline__ cx<T> bsub(cx<T> a, cx<T> b) { return a - b; }
__device__ __forceinline__ df64 df64_add_unnormalised(df64 x, df64 y) {
  const df64 s = two_sum(x.hi, y.hi);
  return {s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo))};
}
template <> __device__ __forceinline__ cx<df64> badd(cx<df64> a, cx<df64> b) {
  return {df64_add_unnormalised(a.r, b.r), df64_add_unnormalised(a.i, b.i)};
}
template <> __device__ __forceinline__ cx<df64> bsub(cx<df64> a, cx<df64> b) {
  return {df64_add_unnormalised(a.r, -b.r), df64_add_unnormalised(a.i, -b.i)};
}

// ---------------- register DFTs (R points, forward sign -1 or inverse sign +1) ----------------
template <typename T, bool INV> __device__ __forceinline__ cx<T> mul_mi(cx<T> a) {
  // forward: multiply by -i; inverse: by +i
  return INV ? cx<T>{-a.i, a.r} : cx<T>{a.i, -a.r};
}

template <typename T, bool INV> __device__ __forceinline__ void dft2(cx<T> *v) {
  const cx<T> a = v[0], b = v[1];
  v[0] = badd(a, b);
  v[1] = bsub(a, b);
}

template <typename T, bool INV> __device__ __forceinline__ void dft3(cx<T> *v) {
  const T h = kconst<T>(0.86602540378443864676);  // sqrt(3)/2
  const cx<T> s = v[1] + v[2], d = v[1] - v[2];
  const T half = kconst<T>(0.5);
  const cx<T> a = {v[0].r - half * s.r, v[0].i - half * s.i};
  const cx<T> b = scale(mul_mi<T, INV>(d), h);  // forward: -i (sqrt3/2) (x1 - x2)
  v[0] = v[0] + s;
  v[1] = a + b;
  v[2] = a - b;
}

template <typename T, bool INV> __device__ __forceinline__ void dft4(cx<T> *v) {
  const cx<T> s02 = badd(v[0], v[2]), d02 = bsub(v[0], v[2]), s13 = badd(v[1], v[3]);
  const cx<T> d13 = mul_mi<T, INV>(bsub(v[1], v[3]));
  v[0] = badd(s02, s13);
  v[2] = bsub(s02, s13);
  v[1] = badd(d02, d13);
  v[3] = bsub(d02, d13);
}

template <typename T, bool INV> __device__ __forceinline__ void dft5(cx<T> *v) {
  const T c1 = kconst<T>(0.30901699437494742410), c2 = kconst<T>(-0.80901699437494742410);  // cos 2pi/5, 4pi/5
  const T s1 = kconst<T>(0.95105651629515357212), s2 = kconst<T>(0.58778525229247312917);   // sin 2pi/5, 4pi/5
  const cx<T> a1 = v[1] + v[4], b1 = v[1] - v[4], a2 = v[2] + v[3], b2 = v[2] - v[3];
  const cx<T> x0 = v[0];
  v[0] = x0 + a1 + a2;
  const cx<T> r1 = {x0.r + c1 * a1.r + c2 * a2.r, x0.i + c1 * a1.i + c2 * a2.i};
  const cx<T> r2 = {x0.r + c2 * a1.r + c1 * a2.r, x0.i + c2 * a1.i + c1 * a2.i};
  // forward: y1 = r1 - i(s1 b1 + s2 b2), y4 = r1 + i(...); y2 = r2 - i(s2 b1 - s1 b2), y3 = r2 + i(...)
  const cx<T> q1 = mul_mi<T, INV>(cx<T>{s1 * b1.r + s2 * b2.r, s1 * b1.i + s2 * b2.i});
  const cx<T> q2 = mul_mi<T, INV>(cx<T>{s2 * b1.r - s1 * b2.r, s2 * b1.i - s1 * b2.i});
  v[1] = r1 + q1;
  v[4] = r1 - q1;
  v[2] = r2 + q2;
  v[3] = r2 - q2;
}

template <typename T, bool INV> __device__ __forceinline__ void dft8(cx<T> *v) {
  cx<T> e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
  dft4<T, INV>(e);
  dft4<T, INV>(o);
  const T h = kconst<T>(0.70710678118654752440);  // 1/sqrt(2)
  // twiddles w8^k, k = 0..3 (forward w8 = (1 - i)/sqrt 2)
  const cx<T> o1 = INV ? cx<T>{h * (o[1].r - o[1].i), h * (o[1].r + o[1].i)}
                       : cx<T>{h * (o[1].r + o[1].i), h * (o[1].i - o[1].r)};
  const cx<T> o2 = mul_mi<T, INV>(o[2]);
  const cx<T> o3 = INV ? cx<T>{-h * (o[3].r + o[3].i), h * (o[3].r - o[3].i)}
                       : cx<T>{h * (o[3].i - o[3].r), -h * (o[3].r + o[3].i)};
  v[0] = badd(e[0], o[0]);
  v[4] = bsub(e[0], o[0]);
  v[1] = badd(e[1], o1);
  v[5] = bsub(e[1], o1);
  v[2] = badd(e[2], o2);
  v[6] = bsub(e[2], o2);
  v[3] = badd(e[3], o3);
  v[7] = bsub(e[3], o3);
}

template <typename T, int R, bool INV> __device__ __forceinline__ void dft(cx<T> *v) {
  if constexpr (R == 2) dft2<T, INV>(v);
  else if constexpr (R == 3) dft3<T, INV>(v);
  else if constexpr (R == 4) dft4<T, INV>(v);
  else if constexpr (R == 5) dft5<T, INV>(v);
  else dft8<T, INV>(v);
}

// One stage over every pencil of the tile along tile dimension a (element stride st, length N).
// Work item w -> (ilo, butterfly beta, ihi); the contiguous index ilo varies fastest so that
// consecutive threads touch consecutive shared-memory words.
template <typename T, int R, bool INV>
__device__ __forceinline__ void fft_stage(cx<T> *tile, const cx<T> *tw, int N, int L, int st, int total_items) {
  const int M = L / R;
  const int nb = N / R;       // butterflies per pencil
  const int twstep = N / L;   // w_L^e = w_N^(e N/L)
  for (int w = threadIdx.x; w < total_items; w += blockDim.x) {
    const int ilo = w % st;
    const int rest = w / st;
    const int beta = rest % nb;
    const int ihi = rest / nb;
    const int blk = beta / M, j = beta - blk * M;
    const int base = ilo + st * (N * ihi + blk * L + j);
    cx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = tile[base + st * M * r];
    // (a stage with M = 1 has j = 0 and unit twiddles: no multiplications; M is uniform per stage)
    if constexpr (!INV) {
      dft<T, R, false>(v);
      if (M > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = v[r] * tw[j * r * twstep];
      }
    } else {
      if (M > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = v[r] * conjg(tw[j * r * twstep]);
      }
      dft<T, R, true>(v);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) tile[base + st * M * r] = v[r];
  }
}

template <typename T, bool INV>
__device__ __forceinline__ void fft_stage_any(int R, cx<T> *tile, const cx<T> *tw, int N, int L, int st, int items) {
  switch (R) {
    case 2: fft_stage<T, 2, INV>(tile, tw, N, L, st, items); break;
    case 3: fft_stage<T, 3, INV>(tile, tw, N, L, st, items); break;
    case 4: fft_stage<T, 4, INV>(tile, tw, N, L, st, items); break;
    case 5: fft_stage<T, 5, INV>(tile, tw, N, L, st, items); break;
    default: fft_stage<T, 8, INV>(tile, tw, N, L, st, items); break;
  }
}

// Full forward (DIF, digit-reversed output) or inverse (DIT, natural output) transform along a tile dim.
template <typename T, bool INV>
__device__ __forceinline__ void fft_axis(cx<T> *tile, const cx<T> *tw, const AxisFFT &ax, int st, int tile_elems) {
  const int N = ax.N;
  if (N == 1) return;
  if (!INV) {
    int L = N;
    for (int k = 0; k < ax.nst; ++k) {
      const int R = ax.R[k];
      fft_stage_any<T, false>(R, tile, tw, N, L, st, tile_elems / R);
      __syncthreads();
      L /= R;
    }
  } else {
    int L = 1;
    for (int k = ax.nst - 1; k >= 0; --k) {
      const int R = ax.R[k];
      L *= R;
      fft_stage_any<T, true>(R, tile, tw, N, L, st, tile_elems / R);
      __syncthreads();
    }
  }
}

// The pass kernel. blockIdx.x: tile, blockIdx.y: packed field. Shared memory: the tile, then the
// twiddle tables of the transformed axes.
template <typename T>
__global__ void __launch_bounds__(512) k_fft_pass(T *__restrict__ data, int64_t V, PassDesc pd, FFTTables tb,
                                                 const Ctrl *ctrl, int check_active, int tkid) {
  data += (int64_t)blockIdx.z * 4 * V * 2;
  ctrl += blockIdx.z;
  if (!should_run<T>(ctrl, check_active)) return;
  count_run(ctrl, tkid);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T> *tile = reinterpret_cast<cx<T> *>(smem_raw);
  const int d0 = pd.d[0], d1 = pd.d[1], d2 = pd.d[2];
  const int nel = d0 * d1 * d2;
  cx<T> *twb = tile + nel;
  // twiddles of the transformed axes
  int twoff[2] = {0, 0};
  {
    int off = 0;
    for (int a = 0; a < pd.nax; ++a) {
      const int mu = pd.ax_mu[a];
      const int N = tb.ax[mu].N;
      const cx<T> *src = reinterpret_cast<const cx<T> *>(tb.tw[mu]);
      for (int k = threadIdx.x; k < N; k += blockDim.x) twb[off + k] = src[k];
      twoff[a] = off;
      off += N;
    }
  }
  const int b = blockIdx.x;
  const int64_t base = (int64_t)(b % pd.nb1) * pd.B1 + (int64_t)(b / pd.nb1) * pd.B2;
  T *field = data + (int64_t)blockIdx.y * V * 2;
  // load the tile (consecutive threads read consecutive i0: runs of d0 contiguous elements)
  for (int e = threadIdx.x; e < nel; e += blockDim.x) {
    const int i0 = e % d0, r = e / d0, i1 = r % d1, i2 = r / d1;
    tile[e] = ld(field, base + i0 * pd.g[0] + i1 * pd.g[1] + i2 * pd.g[2]);
  }
  __syncthreads();
  const int tstride[3] = {1, d0, d0 * d1};
  if (pd.mode == 0 || pd.mode == 2) {
    for (int a = 0; a < pd.nax; ++a)
      fft_axis<T, false>(tile, twb + twoff[a], tb.ax[pd.ax_mu[a]], tstride[pd.ax_dim[a]], nel);
  } else {
    for (int a = pd.nax - 1; a >= 0; --a)
      fft_axis<T, true>(tile, twb + twoff[a], tb.ax[pd.ax_mu[a]], tstride[pd.ax_dim[a]], nel);
  }
  if (pd.mode == 2) {
    // filter: w = p2max / (V p2(k)) at every position; the site index gives the (digit-reversed)
    // position along each lattice axis.
    for (int e = threadIdx.x; e < nel; e += blockDim.x) {
      const int i0 = e % d0, r = e / d0, i1 = r % d1, i2 = r / d1;
      int64_t s = base + i0 * pd.g[0] + i1 * pd.g[1] + i2 * pd.g[2];
      const int px = (int)(s % tb.n[0]);
      s /= tb.n[0];
      const int py = (int)(s % tb.n[1]);
      s /= tb.n[1];
      const int pz = (int)(s % tb.n[2]);
      const int pt = (int)(s / tb.n[2]);
      const double p2 = __ldg(tb.p2part[0] + px) + __ldg(tb.p2part[1] + py) + __ldg(tb.p2part[2] + pz) +
                        __ldg(tb.p2part[3] + pt);
      const T w = p2 == 0.0 ? kconst<T>(0.0) : convert<T>(tb.wscale / p2);
      tile[e] = scale(tile[e], w);
    }
    __syncthreads();
    for (int a = pd.nax - 1; a >= 0; --a)
      fft_axis<T, true>(tile, twb + twoff[a], tb.ax[pd.ax_mu[a]], tstride[pd.ax_dim[a]], nel);
  }
  for (int e = threadIdx.x; e < nel; e += blockDim.x) {
    const int i0 = e % d0, r = e / d0, i1 = r % d1, i2 = r / d1;
    st(field, base + i0 * pd.g[0] + i1 * pd.g[1] + i2 * pd.g[2], tile[e]);
  }
}

}  // namespace lgf
