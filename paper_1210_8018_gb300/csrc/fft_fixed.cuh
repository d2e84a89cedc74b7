// fft_fixed.cuh -- FFT passes specialised at compile time for the common axis lengths
// (8, 16, 24, 32, 48, 64), used by the planner whenever the lattice allows; other lengths use the
// generic passes of fft.cuh. Same mathematics as fft.cuh (in-place mixed-radix DIF forward with a
// digit-reversed spectrum, exact DIT inverse, filter w = p^2_max/(V p^2) fused into the last forward
// pass), with these differences:
//   * every extent, stride inside the tile and radix is a constant, so index arithmetic folds away;
//   * tiles live in shared memory with an odd row pitch and the pencil index varies fastest across
//     threads, so every stage is free of bank conflicts for 8- and 16-byte elements;
//   * each thread issues all of its global loads before any shared-memory store;
//   * the filter pass holds the four packed fields of its columns at once, so the weight of a site
//     is computed once (in the pass's own precision) and applied to all four.
#pragma once
#include "fft.cuh"

namespace lgf {

// Radix plans, identical to the host planner's greedy factorisation (8s first, then 4, 2, 3, 5).
template <int... Rs> struct RadixList {};
template <int N> struct PlanOf;
template <> struct PlanOf<8> { using type = RadixList<8>; };
template <> struct PlanOf<16> { using type = RadixList<8, 2>; };
template <> struct PlanOf<24> { using type = RadixList<8, 3>; };
template <> struct PlanOf<32> { using type = RadixList<8, 4>; };
template <> struct PlanOf<48> { using type = RadixList<8, 2, 3>; };
template <> struct PlanOf<64> { using type = RadixList<8, 8>; };

// One DIF (or inverse DIT) stage of block length L and radix R along a tile axis of length N whose
// elements are `estride` apart; NPEN pencils whose first elements are `pstride` apart.
template <typename T, int N, int L, int R, bool INV, int NPEN, int NT>
__device__ __forceinline__ void fx_stage(cx<T> *tile, const cx<T> *tw, int estride, int pstride) {
  constexpr int M = L / R;
  constexpr int NB = N / R;
  constexpr int TWSTEP = N / L;
  constexpr int ITEMS = NPEN * NB;
#pragma unroll 2
  for (int w = threadIdx.x; w < ITEMS; w += NT) {
    const int pen = w % NPEN;
    const int beta = w / NPEN;
    const int blk = beta / M, j = beta % M;
    cx<T> *p = tile + pen * pstride + (blk * L + j) * estride;
    cx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = p[r * M * estride];
    // (the last stage, M = 1, has j = 0 and unit twiddles: no multiplications)
    if constexpr (!INV) {
      dft<T, R, false>(v);
      if constexpr (M > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = v[r] * tw[j * r * TWSTEP];
      }
    } else {
      if constexpr (M > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = v[r] * conjg(tw[j * r * TWSTEP]);
      }
      dft<T, R, true>(v);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) p[r * M * estride] = v[r];
  }
}

template <typename T, int N, int L, int NPEN, int NT, int R, int... Rest>
__device__ __forceinline__ void fx_forward(cx<T> *tile, const cx<T> *tw, int estride, int pstride) {
  fx_stage<T, N, L, R, false, NPEN, NT>(tile, tw, estride, pstride);
  __syncthreads();
  if constexpr (sizeof...(Rest) > 0) fx_forward<T, N, L / R, NPEN, NT, Rest...>(tile, tw, estride, pstride);
}
template <typename T, int N, int L, int NPEN, int NT, int R, int... Rest>
__device__ __forceinline__ void fx_inverse(cx<T> *tile, const cx<T> *tw, int estride, int pstride) {
  if constexpr (sizeof...(Rest) > 0) fx_inverse<T, N, L / R, NPEN, NT, Rest...>(tile, tw, estride, pstride);
  fx_stage<T, N, L, R, true, NPEN, NT>(tile, tw, estride, pstride);
  __syncthreads();
}
template <typename T, int N, int NPEN, int NT, bool INV, int... Rs>
__device__ __forceinline__ void fx_axis_impl(RadixList<Rs...>, cx<T> *tile, const cx<T> *tw, int estride,
                                             int pstride) {
  if constexpr (!INV) fx_forward<T, N, N, NPEN, NT, Rs...>(tile, tw, estride, pstride);
  else fx_inverse<T, N, N, NPEN, NT, Rs...>(tile, tw, estride, pstride);
}
template <typename T, int N, int NPEN, int NT, bool INV>
__device__ __forceinline__ void fx_axis(cx<T> *tile, const cx<T> *tw, int estride, int pstride) {
  fx_axis_impl<T, N, NPEN, NT, INV>(typename PlanOf<N>::type{}, tile, tw, estride, pstride);
}

template <typename T, int N> __device__ __forceinline__ void load_twiddles(cx<T> *dst, const void *src) {
  const cx<T> *s = reinterpret_cast<const cx<T> *>(src);
  for (int k = threadIdx.x; k < N; k += blockDim.x) dst[k] = s[k];
}


// ---------------------------------------------------------------------------------------------
// xy plane pass: the 2D transform of one (z, t) plane of one packed field. Tile [NY][NX] with row pitch
// NX + 1. blockIdx.x = plane (ntiles = gridDim.x planes), blockIdx.y = field.
// ---------------------------------------------------------------------------------------------
template <typename T, int NX, int NY, bool INV, int NT>
__global__ void __launch_bounds__(NT) k_fx_plane(T *__restrict__ data, int64_t V, FFTTables tb, const Ctrl *ctrl,
                                                int check_active, int tkid, int ntiles) {
  (void)ntiles;
  data += (int64_t)blockIdx.z * 4 * V * 2;
  ctrl += blockIdx.z;
  if (!should_run<T>(ctrl, check_active)) return;
  count_run(ctrl, tkid);
  constexpr int P = NX + 1;
  constexpr int NEL = NX * NY;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T> *tile = reinterpret_cast<cx<T> *>(smem_raw);
  cx<T> *twx = tile + NY * P;
  cx<T> *twy = twx + NX;
  load_twiddles<T, NX>(twx, tb.tw[0]);
  load_twiddles<T, NY>(twy, tb.tw[1]);
  const cx<T> *src = reinterpret_cast<const cx<T> *>(data + (int64_t)blockIdx.y * V * 2) + (int64_t)blockIdx.x * NEL;
  constexpr int PER = (NEL + NT - 1) / NT;
  cx<T> reg[PER];
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int e = threadIdx.x + k * NT;
    if (e < NEL) {
      reg[k] = from_vec<T>(__ldg(reinterpret_cast<const typename vec2<T>::type *>(src) + e));
    }
  }
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int e = threadIdx.x + k * NT;
    if (e < NEL) tile[(e / NX) * P + (e % NX)] = reg[k];
  }
  __syncthreads();
  if (!INV) {
    fx_axis<T, NX, NY, NT, false>(tile, twx, 1, P);  // along x: pencils are rows
    fx_axis<T, NY, NX, NT, false>(tile, twy, P, 1);  // along y: pencils are columns
  } else {
    fx_axis<T, NY, NX, NT, true>(tile, twy, P, 1);
    fx_axis<T, NX, NY, NT, true>(tile, twx, 1, P);
  }
  cx<T> *dst = reinterpret_cast<cx<T> *>(data + (int64_t)blockIdx.y * V * 2) + (int64_t)blockIdx.x * NEL;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int e = threadIdx.x + k * NT;
    if (e < NEL) {
      reinterpret_cast<typename vec2<T>::type *>(dst)[e] = to_vec<T>(tile[(e / NX) * P + (e % NX)]);
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Column pass along one lattice axis of length N (z or t): a tile of N rows (row stride `rstride`
// complex elements) by C contiguous columns, pitch C + 1. Tile b covers columns (b % ncb) * C .. + C of
// outer slice b / ncb (outer stride `ostride`); the pass has ntiles tiles.
//   Where prefetch_tiles() (fft_dispatch.h) says so, blocks loop over tiles b, b + gridDim.x, ... (the
//   planner launches one wave of blocks), and while a tile is transformed in shared memory its successor's
//   elements are already being loaded into registers, so the global loads of one tile overlap the
//   butterflies and the stores of the previous one. Otherwise every block takes tile blockIdx.x.
//   MODE 0: forward (one field per block, blockIdx.y = field)
//   MODE 1: inverse (one field per block)
//   MODE 2: forward + filter + inverse, FPB fields per block (blockIdx.y selects the group of FPB
//           fields): with FPB = 4 the weight of a site is computed once for all four fields (worth it
//           when a weight is expensive, as in df64); in float FPB = 1 keeps the tiles small. This pass
//           must be the last axis (t), so that the columns enumerate x, y, z.
// ---------------------------------------------------------------------------------------------
template <typename T, int N, int C, int MODE, int NT, int FPB = 4>
__global__ void __launch_bounds__(NT) k_fx_cols(T *__restrict__ data, int64_t V, int64_t rstride, int ncb,
                                               int64_t ostride, FFTTables tb, const Ctrl *ctrl, int check_active,
                                               int tkid, int twmu, int ntiles) {
  if constexpr (prefetch_tiles<T, 2, MODE>()) {
  data += (int64_t)blockIdx.z * 4 * V * 2;
  ctrl += blockIdx.z;
  if (!should_run<T>(ctrl, check_active)) return;
  count_run(ctrl, tkid);
  constexpr int P = C + 1;
  constexpr int NF = MODE == 2 ? FPB : 1;
  constexpr int TILE = N * P;
  constexpr int NEL = N * C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T> *tile = reinterpret_cast<cx<T> *>(smem_raw);
  cx<T> *tw = tile + NF * TILE;
  __shared__ T sxyz[MODE == 2 ? C : 1];
  __shared__ T srow[MODE == 2 ? N : 1];
  load_twiddles<T, N>(tw, tb.tw[twmu]);
  if constexpr (MODE == 2) {
    for (int n = threadIdx.x; n < N; n += NT) srow[n] = convert<T>(__ldg(tb.p2part[3] + n));
  }
  using V2 = typename vec2<T>::type;
  constexpr int PER = (NEL + NT - 1) / NT;
  auto base_of = [&](int bb) { return (int64_t)(bb % ncb) * C + (int64_t)(bb / ncb) * ostride; };
  auto field_of = [&](int f) { return MODE == 2 ? (int)blockIdx.y * FPB + f : (int)blockIdx.y; };
  V2 reg[NF][PER];
  auto fetch = [&](int bb) {
    const int64_t base = base_of(bb);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const V2 *src = reinterpret_cast<const V2 *>(data + (int64_t)field_of(f) * V * 2);
#pragma unroll
      for (int k = 0; k < PER; ++k) {
        const int e = threadIdx.x + k * NT;
        if (e < NEL) reg[f][k] = __ldg(src + base + (e / C) * rstride + (e % C));
      }
    }
  };
  constexpr bool kPrefetch = prefetch_tiles<T, 2, MODE>();
  int b = blockIdx.x;
  if (kPrefetch && b < ntiles) fetch(b);
  for (; b < ntiles; b += gridDim.x) {
    if (!kPrefetch) fetch(b);
    const int64_t col0 = (int64_t)(b % ncb) * C;
    const int64_t base = base_of(b);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
#pragma unroll
      for (int k = 0; k < PER; ++k) {
        const int e = threadIdx.x + k * NT;
        if (e < NEL) tile[f * TILE + (e / C) * P + (e % C)] = from_vec<T>(reg[f][k]);
      }
    }
    if constexpr (MODE == 2) {
      // weight of each (row, column): w = p2max / (V (p2_xyz(column) + p2_t(row))), 0 at k = 0
      for (int c = threadIdx.x; c < C; c += NT) {
        const int64_t q = col0 + c;
        const int x = (int)(q % tb.n[0]);
        const int64_t r = q / tb.n[0];
        const int y = (int)(r % tb.n[1]);
        const int z = (int)(r / tb.n[1]);
        sxyz[c] = convert<T>(__ldg(tb.p2part[0] + x) + __ldg(tb.p2part[1] + y) + __ldg(tb.p2part[2] + z));
      }
    }
    __syncthreads();
    if (kPrefetch && b + (int)gridDim.x < ntiles) fetch(b + gridDim.x);  // in flight during the transform
    // along the rows: element stride P, pencils (columns) stride 1; the fields are stacked, TILE apart
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      if (MODE == 1) fx_axis<T, N, C, NT, true>(tile + f * TILE, tw, P, 1);
      else fx_axis<T, N, C, NT, false>(tile + f * TILE, tw, P, 1);
    }
    if constexpr (MODE == 2) {
      const T wscale = convert<T>(tb.wscale);
      const T zero = kconst<T>(0.0);
      for (int e = threadIdx.x; e < NEL; e += NT) {
        const int n = e / C, c = e % C;
        const T p2 = sxyz[c] + srow[n];
        const T w = p2 == zero ? zero : wscale / p2;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          cx<T> &v = tile[f * TILE + n * P + c];
          v = scale(v, w);
        }
      }
      __syncthreads();
#pragma unroll
      for (int f = 0; f < NF; ++f) fx_axis<T, N, C, NT, true>(tile + f * TILE, tw, P, 1);
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      V2 *dst = reinterpret_cast<V2 *>(data + (int64_t)field_of(f) * V * 2);
      for (int e = threadIdx.x; e < NEL; e += NT) {
        const int n = e / C, c = e % C;
        dst[base + n * rstride + c] = to_vec<T>(tile[f * TILE + n * P + c]);
      }
    }
    __syncthreads();
  }
  } else {
  data += (int64_t)blockIdx.z * 4 * V * 2;
  ctrl += blockIdx.z;
  if (!should_run<T>(ctrl, check_active)) return;
  count_run(ctrl, tkid);
  constexpr int P = C + 1;
  constexpr int NF = MODE == 2 ? FPB : 1;
  constexpr int TILE = N * P;
  constexpr int NEL = N * C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T> *tile = reinterpret_cast<cx<T> *>(smem_raw);
  cx<T> *tw = tile + NF * TILE;
  load_twiddles<T, N>(tw, tb.tw[twmu]);
  const int b = blockIdx.x;
  const int64_t col0 = (int64_t)(b % ncb) * C;
  const int64_t base = col0 + (int64_t)(b / ncb) * ostride;
  constexpr int PER = (NEL + NT - 1) / NT;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const int field = MODE == 2 ? (int)blockIdx.y * FPB + f : (int)blockIdx.y;
    const cx<T> *src = reinterpret_cast<const cx<T> *>(data + (int64_t)field * V * 2);
    cx<T> reg[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int e = threadIdx.x + k * NT;
      if (e < NEL) {
        const int n = e / C, c = e % C;
        reg[k] = from_vec<T>(__ldg(reinterpret_cast<const typename vec2<T>::type *>(src) + base + n * rstride + c));
      }
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int e = threadIdx.x + k * NT;
      if (e < NEL) tile[f * TILE + (e / C) * P + (e % C)] = reg[k];
    }
  }
  __syncthreads();
  // along the rows: element stride P, pencils (columns) stride 1; the four fields are stacked, so
  // they form NF*C pencils whose bases are TILE apart: handle each field in turn.
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    if (MODE == 1) fx_axis<T, N, C, NT, true>(tile + f * TILE, tw, P, 1);
    else fx_axis<T, N, C, NT, false>(tile + f * TILE, tw, P, 1);
  }
  if constexpr (MODE == 2) {
    // weight of each (row, column): w = p2max / (V (p2_xyz(column) + p2_t(row))), 0 at k = 0
    __shared__ T sxyz[C];
    __shared__ T srow[N];
    for (int c = threadIdx.x; c < C; c += NT) {
      const int64_t q = col0 + c;
      const int x = (int)(q % tb.n[0]);
      const int64_t r = q / tb.n[0];
      const int y = (int)(r % tb.n[1]);
      const int z = (int)(r / tb.n[1]);
      sxyz[c] = convert<T>(__ldg(tb.p2part[0] + x) + __ldg(tb.p2part[1] + y) + __ldg(tb.p2part[2] + z));
    }
    for (int n = threadIdx.x; n < N; n += NT) srow[n] = convert<T>(__ldg(tb.p2part[3] + n));
    __syncthreads();
    const T wscale = convert<T>(tb.wscale);
    const T zero = kconst<T>(0.0);
    for (int e = threadIdx.x; e < NEL; e += NT) {
      const int n = e / C, c = e % C;
      const T p2 = sxyz[c] + srow[n];
      const T w = p2 == zero ? zero : wscale / p2;
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        cx<T> &v = tile[f * TILE + n * P + c];
        v = scale(v, w);
      }
    }
    __syncthreads();
#pragma unroll
    for (int f = 0; f < NF; ++f) fx_axis<T, N, C, NT, true>(tile + f * TILE, tw, P, 1);
  }
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const int field = MODE == 2 ? (int)blockIdx.y * FPB + f : (int)blockIdx.y;
    cx<T> *dst = reinterpret_cast<cx<T> *>(data + (int64_t)field * V * 2);
    for (int e = threadIdx.x; e < NEL; e += NT) {
      const int n = e / C, c = e % C;
      reinterpret_cast<typename vec2<T>::type *>(dst)[base + n * rstride + c] = to_vec<T>(tile[f * TILE + n * P + c]);
    }
  }
  }
}

// ---------------------------------------------------------------------------------------------
// xy plane pass for 64 x 64 planes in float, the operations of k_fx_plane<T, 64, 64, INV> in the same order
// with the data in registers (512 threads, eight elements each):
//   x phase: thread (j, y) = (threadIdx.x % 8, threadIdx.x / 8) holds elements j + 8r (first radix-8
//   stage, twiddles w^(j r)) and then 8j + r (second stage) of row y; the eight threads of a row are
//   lanes of one warp, so their exchange needs only __syncwarp;
//   y phase: thread (x, jy) = (threadIdx.x % 64, threadIdx.x / 64) holds rows jy + 8r and then 8 jy + r of
//   column x; its exchange goes through the block.
// The forward pass runs x then y; the inverse runs y then x, each axis's two stages in the order of
// k_fx_plane's inverse (unit-twiddle stage first, conjugate twiddles before the second radix 8). Global
// loads and stores are 64-byte (x phase) or 256-byte (y phase) runs. The tile (row pitch 72, elements of a
// row permuted within groups of 8 by col ^ (col / 8 % 8)) serves both phases without bank conflicts.
// Measured at 64^4: 0.204 ms forward and 0.216 ms inverse, against 0.221 ms for the tile passes.
// ---------------------------------------------------------------------------------------------
template <typename T, bool INV>
__global__ void __launch_bounds__(512, 3) k_fx_plane64(T *__restrict__ data, int64_t V, FFTTables tb, const Ctrl *ctrl,
                                                      int check_active, int tkid, int ntiles) {
  constexpr int N = 64, R = 8, P = 72;
  static_assert(std::is_same<T, float>::value, "float pass");
  (void)ntiles;
  data += (int64_t)blockIdx.z * 4 * V * 2;
  ctrl += blockIdx.z;
  if (!should_run<T>(ctrl, check_active)) return;
  count_run(ctrl, tkid);
  __shared__ cx<T> tile[N * P];
  auto at = [](int row, int col) { return row * P + (col ^ ((col >> 3) & 7)); };
  using V2 = typename vec2<T>::type;
  V2 *pl = reinterpret_cast<V2 *>(data + (int64_t)blockIdx.y * V * 2) + (int64_t)blockIdx.x * (N * N);
  const cx<T> *twx = reinterpret_cast<const cx<T> *>(tb.tw[0]);
  const cx<T> *twy = reinterpret_cast<const cx<T> *>(tb.tw[1]);
  const int j = threadIdx.x % R, y = threadIdx.x / R;    // x phase
  const int x = threadIdx.x % N, jy = threadIdx.x / N;   // y phase
  cx<T> v[R];
  if constexpr (!INV) {
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = from_vec<T>(__ldg(pl + y * N + j + R * r));
    dft<T, R, false>(v);
#pragma unroll
    for (int r = 1; r < R; ++r) v[r] = v[r] * twx[j * r];
#pragma unroll
    for (int r = 0; r < R; ++r) tile[at(y, j + R * r)] = v[r];
    __syncwarp();
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = tile[at(y, R * j + r)];
    dft<T, R, false>(v);
#pragma unroll
    for (int r = 0; r < R; ++r) tile[at(y, R * j + r)] = v[r];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = tile[at(jy + R * r, x)];
    dft<T, R, false>(v);
#pragma unroll
    for (int r = 1; r < R; ++r) v[r] = v[r] * twy[jy * r];
#pragma unroll
    for (int r = 0; r < R; ++r) tile[at(jy + R * r, x)] = v[r];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = tile[at(R * jy + r, x)];
    dft<T, R, false>(v);
#pragma unroll
    for (int r = 0; r < R; ++r) pl[(R * jy + r) * N + x] = to_vec<T>(v[r]);
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = from_vec<T>(__ldg(pl + (R * jy + r) * N + x));
    dft<T, R, true>(v);
#pragma unroll
    for (int r = 0; r < R; ++r) tile[at(R * jy + r, x)] = v[r];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = tile[at(jy + R * r, x)];
#pragma unroll
    for (int r = 1; r < R; ++r) v[r] = v[r] * conjg(twy[jy * r]);
    dft<T, R, true>(v);
#pragma unroll
    for (int r = 0; r < R; ++r) tile[at(jy + R * r, x)] = v[r];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = tile[at(y, R * j + r)];
    dft<T, R, true>(v);
#pragma unroll
    for (int r = 0; r < R; ++r) tile[at(y, R * j + r)] = v[r];
    __syncwarp();
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = tile[at(y, j + R * r)];
#pragma unroll
    for (int r = 1; r < R; ++r) v[r] = v[r] * conjg(twx[j * r]);
    dft<T, R, true>(v);
#pragma unroll
    for (int r = 0; r < R; ++r) pl[y * N + j + R * r] = to_vec<T>(v[r]);
  }
}

// ---------------------------------------------------------------------------------------------
// t pass with the filter for N = 64 = 8 x 8, C columns per block, one packed field per block (blockIdx.y),
// with the data in registers: the operations of k_fx_cols<T, 64, C, 2> in the same order, so the results
// are the same bits, but two exchanges through shared memory replace the six trips of its tile.
// Thread (c, j) = (threadIdx.x % C, threadIdx.x / C) holds the eight elements of column c that one radix-8
// butterfly combines:
//   rows j + 8r (r = 0..7): forward stage 1 (radix 8 over r, then twiddles w^(j r));
//   exchange: rows 8j + r: forward stage 2 (radix 8, unit twiddles), the filter w = p2max / (V p^2) (0 at
//   p = 0), inverse stage 2 (radix 8);
//   exchange: rows j + 8r again: inverse stage 1 (conjugate twiddles, radix 8), stored.
// Each cell of the exchange buffer is read after the first exchange by the thread that writes it for the
// second, so one buffer serves both. Five resident blocks per SM (48 registers) were measured best at 64^4:
// 0.229 ms per pass against 0.264 ms for the tile pass; blocks that loop over tiles and load the next one
// during the transform (one wave, 64 or 80 registers) took 0.231 ms.
// ---------------------------------------------------------------------------------------------
template <typename T, int C, int NT>
__global__ void __launch_bounds__(NT, 5) k_fx_tfilter64(T *__restrict__ data, int64_t V, int64_t rstride, int ncb,
                                                       int64_t ostride, FFTTables tb, const Ctrl *ctrl,
                                                       int check_active, int tkid, int twmu, int ntiles) {
  constexpr int N = 64, R = 8;
  static_assert(NT == C * R, "eight threads per column");
  static_assert(std::is_same<T, float>::value, "float pass");
  data += (int64_t)blockIdx.z * 4 * V * 2;
  ctrl += blockIdx.z;
  if (!should_run<T>(ctrl, check_active)) return;
  count_run(ctrl, tkid);
  __shared__ cx<T> xs[N][C];
  __shared__ T sxyz[C];
  __shared__ T srow[N];
  using V2 = typename vec2<T>::type;
  const int c = threadIdx.x % C, j = threadIdx.x / C;
  V2 *fld = reinterpret_cast<V2 *>(data + (int64_t)blockIdx.y * V * 2);
  auto col0_of = [&](int bb) { return (int64_t)(bb % ncb) * C; };
  auto base_of = [&](int bb) { return col0_of(bb) + (int64_t)(bb / ncb) * ostride + c; };
  cx<T> v[R];
  auto fetch = [&](int bb) {
    const int64_t base = base_of(bb);
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = from_vec<T>(__ldg(fld + base + (int64_t)(j + R * r) * rstride));
  };
  if (threadIdx.x < N) srow[threadIdx.x] = convert<T>(__ldg(tb.p2part[3] + threadIdx.x));
  const cx<T> *tw = reinterpret_cast<const cx<T> *>(tb.tw[twmu]);
  // one tile per block (the planner launches ntiles blocks); written as a loop that runs once, the form
  // in which the compiler keeps the kernel in 48 registers without spilling
  int b = blockIdx.x;
  if (b < ntiles) fetch(b);
  for (; b < ntiles; b += ntiles) {
    const int64_t base = base_of(b);
    // weight of each (row, column): w = p2max / (V (p2_xyz(column) + p2_t(row))), 0 at k = 0
    if (threadIdx.x < C) {
      const int64_t q = col0_of(b) + threadIdx.x;
      const int x = (int)(q % tb.n[0]);
      const int64_t rr = q / tb.n[0];
      const int y = (int)(rr % tb.n[1]);
      const int z = (int)(rr / tb.n[1]);
      sxyz[threadIdx.x] = convert<T>(__ldg(tb.p2part[0] + x) + __ldg(tb.p2part[1] + y) + __ldg(tb.p2part[2] + z));
    }
    dft<T, R, false>(v);
#pragma unroll
    for (int r = 1; r < R; ++r) v[r] = v[r] * tw[j * r];
#pragma unroll
    for (int r = 0; r < R; ++r) xs[j + R * r][c] = v[r];
    __syncthreads();
    cx<T> u[R];
#pragma unroll
    for (int r = 0; r < R; ++r) u[r] = xs[R * j + r][c];
    dft<T, R, false>(u);
    {
      const T wscale = convert<T>(tb.wscale);
      const T zero = kconst<T>(0.0);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const T p2 = sxyz[c] + srow[R * j + r];
        const T w = p2 == zero ? zero : wscale / p2;
        // rounded products, as the tile pass stores them: not contracted into the sums of the inverse radix 8
        u[r] = {__fmul_rn(u[r].r, w), __fmul_rn(u[r].i, w)};
      }
    }
    dft<T, R, true>(u);
#pragma unroll
    for (int r = 0; r < R; ++r) xs[R * j + r][c] = u[r];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; ++r) u[r] = xs[j + R * r][c];
#pragma unroll
    for (int r = 1; r < R; ++r) u[r] = u[r] * conjg(tw[j * r]);
    dft<T, R, true>(u);
#pragma unroll
    for (int r = 0; r < R; ++r) fld[base + (int64_t)(j + R * r) * rstride] = to_vec<T>(u[r]);
  }
}

}  // namespace lgf
